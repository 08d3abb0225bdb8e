"""sd_expect_noalloc: the expectation value for callers that cannot allocate
device memory (a fixed budget owned by another allocator, or a loop that
must not pay cudaMalloc's implicit synchronisation).  Its scratch lives in a
static device array, so it must give what sd_expect gives, call after call,
with nothing allocated, and what the CPU oracle gives.  Collected last so
that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

from workloads import random_klocal, heisenberg_lattice

pytestmark = pytest.mark.gpu


def _call(lib, N, n, t, code, ox, oz, oc, stream):
    out = ctypes.c_double(float("nan"))
    st = lib.sd_expect_noalloc(n, ctypes.c_void_p(t.data_ptr()), code, len(oc),
                               ox.ctypes.data_as(N.P_u64), oz.ctypes.data_as(N.P_u64),
                               oc.ctypes.data_as(N.P_dbl), ctypes.byref(out), stream)
    return st, out.value


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_expect_matches_sd_expect(dtype):
    """Calls in a row with observables of 25, 3 and again 25 terms (a call
    that follows a larger one, and one that follows a smaller one, on the
    shared scratch array) each agree with the existing entry point sd_expect
    and with the CPU oracle; after a first call (which loads the module and
    its device array) the device's free memory does not move."""
    import torch
    import oracle
    import paper_2206_11664_gb300 as sd
    from paper_2206_11664_gb300 import _native as N
    lib = N.load()
    rng = np.random.default_rng(808)
    tol = 1e-12 if dtype == "c128" else 1e-5
    cdt = torch.complex128 if dtype == "c128" else torch.complex64
    code = N.SD_C128 if dtype == "c128" else N.SD_C64
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n in (6, 17):
        big = random_klocal(n, 25, rng, weights=(1, 2, 3))      # X, Y and Z-only terms
        small = random_klocal(n, 3, rng, weights=(1, 2))
        v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
        v /= np.linalg.norm(v)
        t = torch.from_numpy(v).to(cdt).cuda()
        host = t.cpu().numpy().astype(np.complex128)            # the state as stored on the device
        checks = []
        for h in (big, small):
            obs = (np.ascontiguousarray(h.x, np.uint64), np.ascontiguousarray(h.z, np.uint64),
                   np.ascontiguousarray(h.c, np.float64))
            ref = sd.Simulator(h.n, h.x, h.z, h.c).plan().expect(t, obs)   # the existing entry point
            want = oracle.expect(host, *obs)
            assert abs(ref - want) <= tol * max(1.0, abs(want))
            checks.append((obs, ref, want))
        st, _ = _call(lib, N, n, t, code, *checks[0][0], stream)     # warm-up call
        assert st == N.SD_OK, lib.sd_last_error(None)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        allocated_before = torch.cuda.memory_allocated()
        for obs, ref, want in (checks[0], checks[1], checks[0], checks[1]):
            st, got = _call(lib, N, n, t, code, *obs, stream)
            assert st == N.SD_OK, lib.sd_last_error(None)
            assert abs(got - ref) <= tol * max(1.0, abs(ref)), (got, ref)
            assert abs(got - want) <= tol * max(1.0, abs(want)), (got, want)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.cuda.memory_allocated() == allocated_before


def test_noalloc_rejects_too_many_terms():
    import torch
    from paper_2206_11664_gb300 import _native as N
    lib = N.load()
    h = heisenberg_lattice(2, 3)
    t = torch.zeros(1 << h.n, dtype=torch.complex128, device="cuda")
    m = 4097
    ox = np.zeros(m, np.uint64)
    oz = np.ones(m, np.uint64)
    oc = np.ones(m)
    st, _ = _call(lib, N, h.n, t, N.SD_C128, ox, oz, oc,
                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == N.SD_EINVAL
    assert b"at most 4096" in lib.sd_last_error(None)
