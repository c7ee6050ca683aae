"""The schedule of the GPU's coarsest inverse, checked on CPU: block sweeps
(Gauss-Jordan elimination without pivoting on an SPD matrix) over 32-row
pivot blocks of the lower triangle, with the padding to a multiple of 32, the
panel (U = S_:P, U S_PP^-1), the tile update in which the next pivot tile is
inverted from its updated values, and the software-pipelined 32 x 32 pivot
inverse (column k+1 and its reciprocal formed during step k).  This models the
kernels' arithmetic order in numpy; the kernels themselves are checked
against the oracle by the GPU tests."""
import numpy as np
import pytest


def pivot_inverse(m):
    """32 scalar sweeps of a 32 x 32 SPD block, pipelined as on the GPU."""
    m = m.copy()
    n = 32
    ck = np.zeros((2, n))
    cs = np.zeros((2, n))
    sdk = np.zeros(2)
    d = m[0, 0]
    ck[0] = m[:, 0]
    cs[0] = ck[0] / d
    sdk[0] = 1.0 / d
    lower = [(i, j) for i in range(n) for j in range(i + 1)]
    for k in range(n):
        cur, nxt = k & 1, (k & 1) ^ 1
        new = m.copy()
        if k + 1 < n:
            kp = k + 1
            col = np.zeros(n)
            for lane in range(n):
                a, b = max(lane, kp), min(lane, kp)
                v = cs[cur][a] if b == k else m[a, b] - ck[cur][a] * cs[cur][b]
                new[a, b] = v
                col[lane] = v
            assert col[kp] > 0
            ck[nxt], cs[nxt], sdk[nxt] = col, col / col[kp], 1.0 / col[kp]
        for i, j in lower:
            if i == k + 1 or j == k + 1:
                continue
            if i == k and j == k:
                v = -sdk[cur]
            elif i == k:
                v = cs[cur][j]
            elif j == k:
                v = cs[cur][i]
            else:
                v = m[i, j] - ck[cur][i] * cs[cur][j]
            new[i, j] = v
        m = new
    out = np.zeros((n, n))
    for i, j in lower:
        out[i, j] = out[j, i] = -m[i, j]
    return out


def sym(S, i, j):
    return S[i, j] if i >= j else S[j, i]


def block_sweep_inverse(A):
    n = A.shape[0]
    nbk = (n + 31) // 32
    npad = 32 * nbk
    S = np.zeros((npad, npad))
    S[:n, :n] = A
    for i in range(n, npad):
        S[i, i] = 1.0
    blk = lambda S, P: np.array([[sym(S, P * 32 + i, P * 32 + j) for j in range(32)] for i in range(32)])
    Dinv = pivot_inverse(blk(S, 0))
    for P in range(nbk):
        Uo = np.array([[sym(S, r, P * 32 + k) for k in range(32)] for r in range(npad)])
        Uh = Uo @ Dinv
        new = S.copy()
        for I in range(nbk):
            for J in range(I + 1):
                for r in range(I * 32, I * 32 + 32):
                    for c in range(J * 32, J * 32 + 32):
                        if I == P and J == P:
                            new[r, c] = -Dinv[r - P * 32, c - P * 32]
                        elif J == P:
                            new[r, c] = Uh[r, c - P * 32]
                        elif I == P:
                            new[r, c] = Uh[c, r - P * 32]
                        else:
                            new[r, c] = S[r, c] - Uh[r] @ Uo[c]
        S = new
        if P + 1 < nbk:
            Dinv = pivot_inverse(blk(S, P + 1))
    return np.array([[-sym(S, i, j) for j in range(n)] for i in range(n)])


@pytest.mark.parametrize("n", [1, 5, 32, 33, 70])
def test_block_sweep_schedule_inverts_spd_matrices(n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B @ B.T / n + np.eye(n)
    X = block_sweep_inverse(A)
    assert np.abs(X @ A - np.eye(n)).max() <= 1e-12
    assert np.array_equal(X, X.T)


def test_pivot_inverse_alone():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((32, 32))
    A = B @ B.T + 32 * np.eye(32)
    assert np.abs(pivot_inverse(A) @ A - np.eye(32)).max() <= 1e-13
