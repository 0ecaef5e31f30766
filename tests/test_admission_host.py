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
// pick_batch over arrays: compatible flags, work, bytes; out: chosen indices and offsets.
int batch(size_t count, double first_work, int max_extra, void* p, const int* compat,
          const double* work, const size_t* bytes, long* chosen, size_t* offs) {
  std::vector<size_t> o;
  const std::vector<size_t> c = gp::sched::pick_batch(
      count, first_work, max_extra, *static_cast<PoolAllocator*>(p),
      [&](size_t k) { return compat[k] != 0; }, [&](size_t k) { return work[k]; },
      [&](size_t k) { return bytes[k]; }, &o);
  for (size_t i = 0; i < c.size(); ++i) { chosen[i] = static_cast<long>(c[i]); offs[i] = o[i]; }
  return static_cast<int>(c.size());
}
// same_batch / batchable on requests given by their fields.
int same(int ka, int da, int pa, int la, int prec_a, int kb, int db, int pb, int lb, int prec_b) {
  gp_request a{}, b{};
  a.kind = 0; a.kernel = ka; a.d = da; a.nprobe = pa; a.nlanczos = la; a.prec = prec_a;
  a.slq_prec = GP_PREC_FP32;
  b.kind = 0; b.kernel = kb; b.d = db; b.nprobe = pb; b.nlanczos = lb; b.prec = prec_b;
  b.slq_prec = GP_PREC_FP32;
  return gp::sched::same_batch(a, b) ? 1 : 0;
}
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
    lib.batch.restype = ctypes.c_int
    lib.batch.argtypes = [ctypes.c_size_t, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p]
    lib.same.restype = ctypes.c_int
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


def _batch(A, first_work, max_extra, pool_bytes, compat, work, nbytes):
    p = A.pool_new(pool_bytes)
    c = np.asarray(compat, dtype=np.int32)
    w = np.asarray(work, dtype=np.float64)
    b = np.asarray(nbytes, dtype=np.uint64)
    chosen = np.zeros(len(w), dtype=np.int64)
    offs = np.zeros(len(w), dtype=np.uint64)
    k = A.batch(len(w), first_work, max_extra, p, c.ctypes.data, w.ctypes.data, b.ctypes.data,
                chosen.ctypes.data, offs.ctypes.data)
    used = A.pool_in_use(p)
    A.pool_free(p)
    return list(chosen[:k]), list(offs[:k]), used


def test_batch_takes_compatible_similar_work_in_increasing_order(A):
    work = [5.0, 1.0, 400.0, 3.0, 2.0, 3.0, 0.01]
    compat = [1, 1, 1, 0, 1, 1, 1]
    chosen, offs, used = _batch(A, 2.0, 8, 1 << 30, compat, work, [1000] * 7)
    # 400 (ratio 200) and 0.01 (ratio 200) are too far from 2; index 3 is not
    # compatible; the rest by increasing work, arrival order among equals.
    assert chosen == [1, 4, 5, 0]
    assert used == 4 * 1024 and len(set(offs)) == 4 and all(o % ALIGN == 0 for o in offs)


def test_batch_respects_max_extra_and_pool(A):
    work = [1.0, 1.5, 2.0, 2.5, 3.0]
    chosen, _, _ = _batch(A, 1.0, 2, 1 << 30, [1] * 5, work, [256] * 5)
    assert chosen == [0, 1]
    # Only two blocks fit: the third and later are left in the queue.
    chosen, _, used = _batch(A, 1.0, 8, 2 * 4096, [1] * 5, work, [4096] * 5)
    assert chosen == [0, 1] and used == 2 * 4096
    chosen, _, _ = _batch(A, 1.0, 0, 1 << 30, [1] * 5, work, [256] * 5)
    assert chosen == []


def test_batch_key(A):
    # kernel, dimension class, nprobe, nlanczos must agree; FP32 products only.
    assert A.same(0, 3, 16, 20, 0, 0, 3, 16, 20, 0) == 1
    assert A.same(0, 6, 16, 20, 0, 0, 8, 16, 20, 0) == 1      # both in the class 5..8
    assert A.same(0, 4, 16, 20, 0, 0, 5, 16, 20, 0) == 0
    assert A.same(0, 3, 16, 20, 0, 1, 3, 16, 20, 0) == 0
    assert A.same(0, 3, 16, 20, 0, 0, 3, 8, 20, 0) == 0
    assert A.same(0, 3, 16, 20, 0, 0, 3, 16, 30, 0) == 0
    assert A.same(0, 3, 16, 20, 4, 0, 3, 16, 20, 4) == 0      # split BF16 products
    assert A.same(0, 3, 63, 20, 0, 0, 3, 63, 20, 0) == 1      # 1 + nprobe = 64
    assert A.same(0, 3, 64, 20, 0, 0, 3, 64, 20, 0) == 0
