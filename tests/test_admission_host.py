"""CPU checks of the request server's host-side scheduling (csrc/admission.h),
built with the host compiler from the same header the server compiles:

  * the pool allocator against a brute-force first-fit model over random
    allocation / release sequences (offsets, alignment, bytes in use, full
    coalescing once everything is released);
  * the admission rule: least work first among the requests that fit, arrival
    order among equal work, the oldest request first once it has waited the
    ageing time (and nothing else while it does not fit);
  * the work measure and the stream priority level in closed form.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_02259_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
ALIGN = 256
AGE_S = 30.0

SHIM = r"""
#include "admission.h"
using gp::sched::PoolAllocator;
extern "C" {
void* pool_new(size_t n) { return new PoolAllocator(n); }
void pool_free(void* p) { delete static_cast<PoolAllocator*>(p); }
int pool_alloc(void* p, size_t b, size_t* off) { return static_cast<PoolAllocator*>(p)->alloc(b, off); }
void pool_release(void* p, size_t off, size_t b) { static_cast<PoolAllocator*>(p)->release(off, b); }
size_t pool_in_use(void* p) { return static_cast<PoolAllocator*>(p)->in_use(); }
size_t pool_extents(void* p) { return static_cast<PoolAllocator*>(p)->free_extents(); }
long pick(size_t count, double now, void* p, const double* work, const double* tsub,
          const size_t* bytes, size_t* off) {
  return gp::sched::pick_next(count, now, *static_cast<PoolAllocator*>(p),
                              [&](size_t k) { return work[k]; }, [&](size_t k) { return tsub[k]; },
                              [&](size_t k) { return bytes[k]; }, off);
}
static gp_request req(int kind, long long n, int nprobe, int nlanczos, int maxit, long long m) {
  gp_request r{};
  r.kind = kind; r.n = n; r.nprobe = nprobe; r.nlanczos = nlanczos; r.cg_maxit = maxit; r.m = m;
  return r;
}
double work_of(int kind, long long n, int nprobe, int nlanczos, int maxit, long long m) {
  return gp::sched::request_work(req(kind, n, nprobe, nlanczos, maxit, m));
}
int level_of(int kind, long long n, int nprobe, int nlanczos, int maxit, long long m, int levels) {
  return gp::sched::priority_level(req(kind, n, nprobe, nlanczos, maxit, m), levels);
}
double age_seconds() { return gp::sched::kAgeSeconds; }
}
"""


@pytest.fixture(scope="module")
def A(tmp_path_factory):
    d = tmp_path_factory.mktemp("adm")
    src = d / "adm.cpp"
    src.write_text(SHIM)
    so = d / "adm.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-I", INCLUDE,
                    str(src), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.pool_new.restype = ctypes.c_void_p
    lib.pool_new.argtypes = [ctypes.c_size_t]
    lib.pool_free.argtypes = [ctypes.c_void_p]
    lib.pool_alloc.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.pool_release.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t]
    lib.pool_in_use.restype = ctypes.c_size_t
    lib.pool_in_use.argtypes = [ctypes.c_void_p]
    lib.pool_extents.restype = ctypes.c_size_t
    lib.pool_extents.argtypes = [ctypes.c_void_p]
    lib.pick.restype = ctypes.c_long
    lib.pick.argtypes = [ctypes.c_size_t, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    lib.work_of.restype = ctypes.c_double
    lib.work_of.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_longlong]
    lib.level_of.argtypes = lib.work_of.argtypes + [ctypes.c_int]
    lib.age_seconds.restype = ctypes.c_double
    return lib


def _up(b):
    return (b + ALIGN - 1) // ALIGN * ALIGN


def _model_first_fit(used, size, b):
    """Lowest offset of a free gap of at least b bytes given the used extents."""
    at = 0
    for o, n in sorted(used.items()):
        if o - at >= b:
            return at
        at = o + n
    return at if size - at >= b else None


def test_age_constant(A):
    assert A.age_seconds() == AGE_S


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pool_allocator_matches_first_fit_model(A, seed):
    rng = np.random.default_rng(seed)
    size = 64 * 1024 * ALIGN
    p = A.pool_new(size)
    used = {}
    try:
        for step in range(3000):
            if used and (rng.random() < 0.45 or len(used) > 60):
                o = list(used)[int(rng.integers(len(used)))]
                n = used.pop(o)
                A.pool_release(p, o, n - int(rng.integers(0, ALIGN)) if n > ALIGN else n)
            else:
                b = int(rng.integers(1, size // 16))
                off = ctypes.c_size_t()
                ok = A.pool_alloc(p, b, ctypes.byref(off))
                want = _model_first_fit(used, size, _up(b))
                if want is None:
                    assert not ok
                else:
                    assert ok and off.value == want and off.value % ALIGN == 0
                    used[off.value] = _up(b)
            assert A.pool_in_use(p) == sum(used.values())
        for o, n in list(used.items()):
            A.pool_release(p, o, n)
        assert A.pool_in_use(p) == 0 and A.pool_extents(p) == 1
        off = ctypes.c_size_t()
        assert A.pool_alloc(p, size, ctypes.byref(off)) and off.value == 0
        assert not A.pool_alloc(p, 1, ctypes.byref(off))
    finally:
        A.pool_free(p)


def _pick(A, pool, now, work, tsub, nbytes):
    work = np.ascontiguousarray(work, dtype=np.float64)
    tsub = np.ascontiguousarray(tsub, dtype=np.float64)
    nb = np.ascontiguousarray(nbytes, dtype=np.uint64)
    off = ctypes.c_size_t(12345)
    i = A.pick(len(work), now, pool, work.ctypes.data, tsub.ctypes.data, nb.ctypes.data,
               ctypes.byref(off))
    return i, off.value


def test_admission_least_work_that_fits(A):
    p = A.pool_new(100 * ALIGN)
    try:
        # Queue in arrival order: work 5, 1, 3, 1 (ties go to the earlier).
        i, off = _pick(A, p, 1.0, [5, 1, 3, 1], [0.0, 0.1, 0.2, 0.3], [ALIGN] * 4)
        assert (i, off) == (1, 0) and A.pool_in_use(p) == ALIGN
        # The least-work request does not fit: the next one that fits starts.
        i, off = _pick(A, p, 1.0, [1, 2, 3], [0.0, 0.1, 0.2], [200 * ALIGN, 150 * ALIGN, 10 * ALIGN])
        assert (i, off) == (2, ALIGN) and A.pool_in_use(p) == 11 * ALIGN
        # Nothing fits: no admission and nothing reserved.
        i, _ = _pick(A, p, 1.0, [1, 2], [0.0, 0.1], [90 * ALIGN, 95 * ALIGN])
        assert i == -1 and A.pool_in_use(p) == 11 * ALIGN
        # Empty queue.
        i, _ = _pick(A, p, 1.0, [], [], [])
        assert i == -1
    finally:
        A.pool_free(p)


def test_admission_aged_request_first(A):
    p = A.pool_new(100 * ALIGN)
    try:
        # The head has waited the ageing time: it starts although it has the most work.
        i, off = _pick(A, p, AGE_S + 1.0, [9e12, 1.0, 2.0], [1.0, 5.0, 6.0], [10 * ALIGN, ALIGN, ALIGN])
        assert (i, off) == (0, 0)
        # Just under the ageing time the least work wins.
        i, _ = _pick(A, p, AGE_S + 0.99, [9e12, 1.0], [1.0, 5.0], [10 * ALIGN, ALIGN])
        assert i == 1
        # An aged head that does not fit holds the queue: nothing else starts.
        used = A.pool_in_use(p)
        i, _ = _pick(A, p, 100.0, [9e12, 1.0], [1.0, 90.0], [95 * ALIGN, ALIGN])
        assert i == -1 and A.pool_in_use(p) == used
    finally:
        A.pool_free(p)


def test_request_work_and_priority_level(A):
    # Loss + gradient: n^2 (1 + p) (maxit + k + 1) entries x columns.
    assert A.work_of(0, 1000, 16, 20, 20, 0) == 1e6 * 17 * 41
    # Defaults: maxit 1000, k 20.
    assert A.work_of(0, 1000, 0, 0, 0, 0) == 1e6 * 1 * 1021
    # Prediction: n^2 maxit + n m.
    assert A.work_of(1, 2000, 0, 0, 50, 10000) == 4e6 * 50 + 2000 * 10000
    # One level per decade of work from 1e10, clamped to the device's levels.
    assert A.level_of(1, 1000, 0, 0, 1, 0, 6) == 0                  # 1e6
    assert A.level_of(1, 100000, 0, 0, 1, 0, 6) == 1                # 1e10
    assert A.level_of(1, 100000, 0, 0, 10, 0, 6) == 2               # 1e11
    assert A.level_of(1, 1000000, 0, 0, 1000, 0, 6) == 5            # 1e15 -> 6 levels
    assert A.level_of(1, 1000000, 0, 0, 1000, 0, 3) == 2            # clamped
    assert A.level_of(1, 1000000, 0, 0, 1000, 0, 1) == 0
