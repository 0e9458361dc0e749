"""CSR matrix of Pauli sums on the GPU (mat(O), Sec. "Matrix Representation")
against the oracle: column j of the dense matrix is the oracle's O applied to
basis state |j>; the CSR holds exactly its nonzero entries (exact zeros from
cancelling terms dropped), columns ascending, values to 1e-15.  n = 20
Heisenberg (the paper's mat(heisenberg(20)) workload): sampled rows against the
oracle and structural properties (Hermitian, expected nonzeros per row)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import qsim
    return qsim


def dense_oracle(n, terms):
    dim = 1 << n
    H = np.zeros((dim, dim), dtype=np.complex128)
    for j in range(dim):
        H[:, j] = oracle.apply_observable(oracle.basis_state(n, j), n, terms)
    return H


def to_dense(rowptr, cols, vals, n):
    rp, c, v = rowptr.cpu().numpy(), cols.cpu().numpy(), vals.cpu().numpy()
    dim = 1 << n
    H = np.zeros((dim, dim), dtype=np.complex128)
    for i in range(dim):
        cc = c[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cc) > 0), i  # ascending, no duplicates
        H[i, cc] = v[rp[i]:rp[i + 1]]
    return H


def cases(n):
    yield "heisenberg", W.heisenberg(n)
    yield "tfim", W.tfim(n, 0.8)
    yield "mixed", [(0.5, ((0, "X"), (1, "Y"))), (-0.5, ((0, "Y"), (1, "X"))), (1.25, ()),
                    (0.3, ((2, "Z"),)), (0.7, ((0, "Y"), (n - 1, "Y"), (2, "X"))), (-0.2, ((1, "Z"), (3, "Z")))]


@pytest.mark.parametrize("n", [4, 7, 9])
def test_csr_matches_dense_oracle(qs, n):
    for name, terms in cases(n):
        rowptr, cols, vals = qs.observable_csr(qs.Observable(terms), n)
        H = to_dense(rowptr, cols, vals, n)
        want = dense_oracle(n, terms)
        assert np.max(np.abs(H - want)) < 1e-15, name
        assert int(rowptr[-1]) == int(np.count_nonzero(want)), name
        assert np.allclose(want, want.conj().T)


def test_heisenberg_20_sampled_rows(qs):
    n = 20
    terms = W.heisenberg(n)
    rowptr, cols, vals = qs.observable_csr(qs.Observable(terms), n)
    rp = rowptr.cpu().numpy()
    # XX + YY on a bond flips it only when its two bits differ: per row, the diagonal
    # (unless every ZZ cancels) plus one entry per anti-aligned bond
    rs = np.random.default_rng(20)
    for i in list(rs.integers(0, 1 << n, 16)) + [0, (1 << n) - 1, 0x55555]:
        i = int(i)
        col = oracle.apply_observable(oracle.basis_state(n, i), n, terms)  # column i = row i (Hermitian)
        nz = np.nonzero(col)[0]
        c = cols[rp[i]:rp[i + 1]].cpu().numpy()
        v = vals[rp[i]:rp[i + 1]].cpu().numpy()
        assert np.array_equal(c, nz), i
        assert np.max(np.abs(v - np.conj(col[nz]))) < 1e-14, i
        bonds = [(k, (k + 1) % n) for k in range(n)]
        anti = sum(((i >> a) & 1) != ((i >> b) & 1) for a, b in bonds)
        diag = sum(1.0 if ((i >> a) & 1) == ((i >> b) & 1) else -1.0 for a, b in bonds)
        assert len(c) == anti + (diag != 0), i
