"""qs_expect_static: expectation values for callers that cannot allocate device
memory (frameworks owning all device memory, loops that must avoid
cudaMalloc/cudaFree, fixed memory budgets).  Its scratch is a fixed device
array inside the library, so this file checks, through the C ABI, that two
calls in a row give the same values as qs_expect (which uses allocated
scratch) and as the FP64 oracle's expectation of the same amplitudes (a
complex64 state is promoted exactly, so both precisions are held to 1e-12),
and that requests larger than the fixed array are rejected.  Collected last on
purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"c64": torch.complex64, "c128": torch.complex128}
TOL = {"c64": 1e-9, "c128": 1e-12}


def _terms(terms):
    from paper_1912_10877_gb300 import _native as N
    arr = (N.PauliTerm * max(1, len(terms)))()
    for i, (c, ops) in enumerate(terms):
        x = z = 0
        for l, p in ops:
            if p in "XY":
                x |= 1 << l
            if p in "ZY":
                z |= 1 << l
        arr[i].coeff, arr[i].x_mask, arr[i].z_mask = c, x, z
    return arr


def _random_terms(n, count, seed):
    rs = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        q = rs.permutation(n)[: rs.integers(1, n + 1)]
        out.append((float(rs.standard_normal()), tuple((int(l), "XYZ"[rs.integers(3)]) for l in q)))
    return out


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import _native as N
    from paper_1912_10877_gb300 import qsim
    return N, qsim


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_static_matches_allocating_entry_point_twice(env, dt):
    N, qs = env
    L = N.lib()
    cases = [(10, 1, _random_terms(10, 20, 1)), (12, 5, W.tfim(12)), (20, 1, W.zz_chain(20) + _random_terms(20, 9, 2)),
             (3, 300, W.heisenberg(3))]
    for n, nreg, terms in cases:
        st = qs.State(n, dtype=TDT[dt], nbatch=nreg)
        st.upload(np.concatenate([W.haar_state(n, seed=r + 7 * n) for r in range(nreg)]))
        ref = st.expect(qs.Observable(terms))
        amps = st.numpy().astype(np.complex128).reshape(nreg, 1 << n)
        want = np.array([oracle.expect(amps[r], n, terms) for r in range(nreg)])
        out = torch.full((nreg,), float("nan"), dtype=torch.float64, device="cuda")
        arr = _terms(terms)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        code = N.QS_C64 if dt == "c64" else N.QS_C128
        for call in range(2):
            out.fill_(float("nan"))
            N.check(L.qs_expect_static(ctypes.c_void_p(st.buffer.data_ptr()), code, n, nreg, arr, len(terms),
                                       ctypes.c_void_p(out.data_ptr()), stream))
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), (n, nreg, call)
            assert np.max(np.abs(got - ref)) < TOL[dt], (n, nreg, call)
            assert np.max(np.abs(got - want)) < 1e-12, (n, nreg, call, np.max(np.abs(got - want)))


def test_static_rejects_oversize_requests(env):
    N, qs = env
    L = N.lib()
    st = qs.State(4, dtype=torch.complex64, nbatch=2000)
    st.reset()
    out = torch.zeros(2000, dtype=torch.float64, device="cuda")
    terms = _terms(W.zz_chain(4) * 11)  # 33 terms x 2000 registers > 65536 partial sums
    rc = L.qs_expect_static(ctypes.c_void_p(st.buffer.data_ptr()), N.QS_C64, 4, 2000, terms, 33,
                            ctypes.c_void_p(out.data_ptr()), None)
    assert rc == N.QS_EINVAL and b"static scratch" in L.qs_last_error()
    rc = L.qs_expect_static(ctypes.c_void_p(st.buffer.data_ptr()), N.QS_C64, 4, 1, _terms(W.zz_chain(4) * 22), 66,
                            ctypes.c_void_p(out.data_ptr()), None)
    assert rc == N.QS_EINVAL
