"""The multigrid cycle the PCG kernel applies, checked as linear algebra on
the CPU (numpy, no GPU and no oracle).

The kernel writes one V(1,1) cycle as one linear map per level:
  x_l = w_l D_l^-1 r_l,  f_l = x_l + w_l D_l^-1 (r_l - A_l x_l),
  r_{l+1} = Q_l^T r_l,   z_l = f_l + Q_l z_{l+1},
with Q_l = (I - w_l D_l^-1 A_l) P_l, and on the level next to the coarsest
z = f + W r with W = Q C^-1 Q^T.  These tests pin that this is the same
operator as the cycle in its textbook order (pre-smoothing, residual,
restriction, coarse solve, prolongation, post-smoothing), that it is
symmetric positive definite, that the set-up's Q, taken in the pattern of
A P, agrees with (I - w D^-1 A) P, and that one cycle applied to a residual
(the one-cycle correction pass of the mixed refinement) never increases the
error's A-norm.
"""
import numpy as np
import pytest


def _spd_block_banded(n, bw, rng):
    """SPD matrix of n 7x7 block rows with block bandwidth bw."""
    m = 7 * n
    B = np.zeros((m, m))
    for i in range(n):
        for j in range(max(0, i - bw), min(n, i + bw + 1)):
            B[7 * i:7 * i + 7, 7 * j:7 * j + 7] = rng.standard_normal((7, 7))
    return B @ B.T + 0.1 * np.eye(m)


def _block_diag_inv(A, n):
    D = np.zeros_like(A)
    for i in range(n):
        s = slice(7 * i, 7 * i + 7)
        D[s, s] = np.linalg.inv(A[s, s])
    return D


def _hierarchy(n0, levels, rng):
    """Operators, D^-1, weights and smoothed prolongations of a hierarchy with
    aggregates of 4 consecutive nodes and random tentative 7x7 blocks."""
    A = [_spd_block_banded(n0, 3, rng)]
    Dinv, w, P, n = [], [], [], [n0]
    for _ in range(levels):
        nl = n[-1]
        Di = _block_diag_inv(A[-1], nl)
        rho = max(abs(np.linalg.eigvals(Di @ A[-1])))
        nc = (nl + 3) // 4
        T = np.zeros((7 * nl, 7 * nc))
        for u in range(nl):
            c = u // 4
            T[7 * u:7 * u + 7, 7 * c:7 * c + 7] = rng.standard_normal((7, 7)) + 3 * np.eye(7)
        Pl = (np.eye(7 * nl) - 4.0 / (3.0 * rho) * Di @ A[-1]) @ T
        Dinv.append(Di)
        w.append(1.0 / rho)
        P.append(Pl)
        A.append(Pl.T @ A[-1] @ Pl)
        n.append(nc)
    return A, Dinv, w, P


def _cycle_textbook(A, Dinv, w, P, l, r):
    L = len(P)
    if l == L:
        return np.linalg.solve(A[L], r)
    x = w[l] * Dinv[l] @ r                          # pre-smoothing from 0
    s = r - A[l] @ x                                # residual
    y = _cycle_textbook(A, Dinv, w, P, l + 1, P[l].T @ s)   # restriction, coarse cycle
    x = x + P[l] @ y                                # prolongation
    return x + w[l] * Dinv[l] @ (r - A[l] @ x)      # post-smoothing


def _cycle_one_map(A, Dinv, w, P, r):
    L = len(P)
    Q = [P[l] - w[l] * Dinv[l] @ A[l] @ P[l] for l in range(L)]
    d = L - 1
    W = Q[d] @ np.linalg.inv(A[L]) @ Q[d].T
    f, rl = [], r
    for l in range(d + 1):                          # way down: f_l and r_{l+1} from r_l
        x = w[l] * Dinv[l] @ rl
        f.append(x + w[l] * Dinv[l] @ (rl - A[l] @ x))
        if l < d:
            rl = Q[l].T @ rl
    z = f[d] + W @ rl                               # the dense level
    for l in range(d - 1, -1, -1):                  # way up
        z = f[l] + Q[l] @ z
    return z


@pytest.mark.parametrize("n0,levels", [(40, 1), (40, 2), (64, 3)])
def test_one_map_cycle_is_the_textbook_cycle(n0, levels):
    rng = np.random.default_rng(n0 + levels)
    A, Dinv, w, P = _hierarchy(n0, levels, rng)
    m = 7 * n0
    M1 = np.column_stack([_cycle_textbook(A, Dinv, w, P, 0, e) for e in np.eye(m)])
    M2 = np.column_stack([_cycle_one_map(A, Dinv, w, P, e) for e in np.eye(m)])
    scale = np.abs(M1).max()
    assert np.abs(M1 - M2).max() <= 1e-10 * scale
    # the preconditioner is symmetric positive definite
    assert np.abs(M2 - M2.T).max() <= 1e-10 * scale
    assert np.linalg.eigvalsh(0.5 * (M2 + M2.T)).min() > 0.0


def test_q_in_the_pattern_of_a_p():
    """Q = (I - w D^-1 A) P is nonzero only where A P is (A has every diagonal
    block, so A P's pattern also contains P's), and its blocks equal
    P_uc - w D_u^-1 (A P)_uc, which is how the set-up forms them."""
    rng = np.random.default_rng(7)
    A, Dinv, w, P = _hierarchy(32, 1, rng)
    AP = A[0] @ P[0]
    Q = P[0] - w[0] * Dinv[0] @ AP
    nb, nc = 32, 8
    for u in range(nb):
        for c in range(nc):
            blk = (slice(7 * u, 7 * u + 7), slice(7 * c, 7 * c + 7))
            if not np.any(AP[blk]):
                assert not np.any(P[0][blk]) and not np.any(Q[blk])
            Du = Dinv[0][7 * u:7 * u + 7, 7 * u:7 * u + 7]
            assert np.allclose(Q[blk], P[0][blk] - w[0] * Du @ AP[blk], rtol=1e-12, atol=1e-12 * np.abs(Q).max())


@pytest.mark.parametrize("n0,levels", [(40, 1), (40, 2), (64, 3)])
def test_one_cycle_correction_contracts(n0, levels):
    """The mixed refinement's correction pass may apply one cycle, x = B r,
    to its residual (a preconditioned Richardson step).  The error after it
    is (I - B A) e, and with the symmetric cycle every eigenvalue of B A lies
    in (0, 1]: the step never increases the A-norm of the error, and it
    shrinks it by the factor 1 - lambda_min(B A) < 1."""
    rng = np.random.default_rng(100 + n0 + levels)
    A, Dinv, w, P = _hierarchy(n0, levels, rng)
    m = 7 * n0
    B = np.column_stack([_cycle_one_map(A, Dinv, w, P, e) for e in np.eye(m)])
    lam = np.sort(np.linalg.eigvals(B @ A[0]).real)
    assert lam[0] > 0.0 and lam[-1] <= 1.0 + 1e-9
    # the same on a residual: the A-norm of the error drops after x = B r
    e = rng.standard_normal(m)
    r = A[0] @ e
    e1 = e - B @ r
    assert e1 @ A[0] @ e1 <= (1.0 - lam[0]) ** 2 * (e @ A[0] @ e) * (1 + 1e-9)
