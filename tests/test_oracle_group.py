"""Pins of the oracle's Sim(3) arithmetic against closed forms and identities
that do not use the oracle's own routines (Sec. IV-F needs exact Jacobians:
automatic differentiation replaces numerical differentiation)."""
import numpy as np
import pytest

import oracle as O
from paper_2603_17201_gb300 import synthetic as syn

RNG = np.random.default_rng(12345)


def rodrigues_quat(omega):
    th = np.linalg.norm(omega)
    if th == 0:
        return np.array([0, 0, 0, 1.0])
    return np.concatenate([np.sin(th / 2) * omega / th, [np.cos(th / 2)]])


def same_pose(a, b, tol):
    qa, qb = a[:4], b[:4]
    if np.dot(qa, qb) < 0:
        qb = -qb
    return np.abs(qa - qb).max() < tol and np.abs(a[4:] - b[4:]).max() < tol * max(1, np.abs(a[4:]).max())


def W_closed(omega, sigma):
    """V matrix W = A I + B w^ + C w^2 from the integral of
    exp(tau (w^ + sigma I)) over tau in [0, 1] (textbook closed form)."""
    th = np.linalg.norm(omega)
    Wh = np.array([[0, -omega[2], omega[1]], [omega[2], 0, -omega[0]], [-omega[1], omega[0], 0]])
    es = np.exp(sigma)
    A = (es - 1) / sigma
    d = sigma ** 2 + th ** 2
    B = (es * (sigma * np.sin(th) - th * np.cos(th)) + th) / (th * d)
    C = (A - (es * (sigma * np.cos(th) + th * np.sin(th)) - sigma) / d) / th ** 2
    return A * np.eye(3) + B * Wh + C * Wh @ Wh


@pytest.mark.parametrize("scale", [1e-9, 1e-6, 1e-3, 0.1, 1.0, 2.5])
def test_log_exp_roundtrip(oracle_mod, scale):
    for _ in range(20):
        xi = RNG.normal(size=7) * scale
        th = np.linalg.norm(xi[:3])
        if th > 3.0:        # log is the principal branch: |omega| < pi
            xi[:3] *= 3.0 / th
        back = O.log(O.exp(xi))
        assert np.abs(back - xi).max() <= 1e-14 * max(1.0, np.abs(xi).max() ** 2)


def test_log_near_pi(oracle_mod):
    for th in [np.pi - 1e-3, np.pi - 1e-7]:
        axis = RNG.normal(size=3)
        axis /= np.linalg.norm(axis)
        xi = np.concatenate([th * axis, RNG.normal(size=3), [0.3]])
        assert np.abs(O.log(O.exp(xi)) - xi).max() < 1e-9


def test_exp_log_roundtrip_poses(oracle_mod):
    for _ in range(50):
        q = RNG.normal(size=4)
        q /= np.linalg.norm(q)
        p = np.concatenate([q, RNG.normal(size=3) * 20, [np.exp(RNG.normal())]])
        assert same_pose(O.exp(O.log(p)), p, 1e-12)


def test_exp_special_cases(oracle_mod):
    # pure rotation: Rodrigues
    om = np.array([0.3, -0.2, 0.9])
    p = O.exp(np.concatenate([om, [0, 0, 0], [0]]))
    assert same_pose(p, np.concatenate([rodrigues_quat(om), [0, 0, 0], [1]]), 1e-15)
    # pure translation: identity W
    u = np.array([1.5, -2.0, 0.25])
    p = O.exp(np.concatenate([[0, 0, 0], u, [0]]))
    assert same_pose(p, np.concatenate([[0, 0, 0, 1], u, [1]]), 1e-15)
    # translation with scale, no rotation: W = (e^s - 1)/s I
    s = 0.7
    p = O.exp(np.concatenate([[0, 0, 0], u, [s]]))
    assert same_pose(p, np.concatenate([[0, 0, 0, 1], (np.exp(s) - 1) / s * u, [np.exp(s)]]), 1e-14)


@pytest.mark.parametrize("omega,sigma", [
    ([0.3, -0.5, 0.8], 0.4), ([1.2, 0.1, -0.7], -1.1), ([2.0, 1.0, 0.5], 2.0),
    ([0.01, 0.02, -0.01], 0.5), ([0.4, 0.1, 0.2], 1e-3),
])
def test_W_matches_closed_form(oracle_mod, omega, sigma):
    omega = np.array(omega, dtype=float)
    assert np.abs(O.W(omega, sigma) - W_closed(omega, sigma)).max() < 1e-12


def test_W_limits(oracle_mod):
    w = np.array([0.3, -0.2, 0.5])
    Wh = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    # theta -> 0: A = (e^s-1)/s, B = ((s-1)e^s+1)/s^2, C = (e^s(s^2-2s+2)-2)/(2 s^3)
    s = 0.8
    tiny = 1e-9 * w
    A = (np.exp(s) - 1) / s
    B = ((s - 1) * np.exp(s) + 1) / s ** 2
    C = (np.exp(s) * (s * s - 2 * s + 2) - 2) / (2 * s ** 3)
    th = np.linalg.norm(tiny)
    Th = Wh * 1e-9
    ref = A * np.eye(3) + B * Th + C * Th @ Th
    assert np.abs(O.W(tiny, s) - ref).max() < 1e-15
    assert th < 1e-8
    # sigma -> 0: A = 1, B = (1-cos)/th^2, C = (th - sin)/th^3
    th = np.linalg.norm(w)
    ref = np.eye(3) + (1 - np.cos(th)) / th ** 2 * Wh + (th - np.sin(th)) / th ** 3 * Wh @ Wh
    assert np.abs(O.W(w, 0.0) - ref).max() < 1e-15
    # both -> 0: A = 1, B = 1/2, C = 1/6
    assert np.abs(O.W(np.zeros(3), 0.0) - np.eye(3)).max() == 0.0


def test_adjoint_identity(oracle_mod):
    # S exp(xi) S^-1 = exp(Adj(S) xi)
    for _ in range(10):
        q = RNG.normal(size=4)
        q /= np.linalg.norm(q)
        S = np.concatenate([q, RNG.normal(size=3) * 5, [np.exp(0.5 * RNG.normal())]])
        xi = RNG.normal(size=7) * 0.3
        lhs = syn.compose(syn.compose(S, O.exp(xi)), syn.inverse(S))
        rhs = O.exp(O.adj(S) @ xi)
        assert same_pose(lhs, rhs, 1e-12)


def test_left_jacobian_fd(oracle_mod):
    # exp(xi + h e_k) exp(xi)^-1 = exp(h J_l e_k + O(h^2)); central differences
    for scale in [0.05, 0.7, 2.0]:
        xi = RNG.normal(size=7) * scale
        J = O.left_jacobian(xi)
        h = 1e-6
        num = np.zeros((7, 7))
        base_inv = syn.inverse(O.exp(xi))
        for k in range(7):
            d = np.zeros(7)
            d[k] = h
            lp = O.log(syn.compose(O.exp(xi + d), base_inv))
            lm = O.log(syn.compose(O.exp(xi - d), base_inv))
            num[:, k] = (lp - lm) / (2 * h)
        assert np.abs(num - J).max() < 1e-7 * max(1.0, np.abs(J).max())
        # ad(xi) xi = 0 implies J_l(xi) xi = xi
        assert np.abs(J @ xi - xi).max() < 1e-13 * max(1, np.abs(xi).max())
        # Adj(exp(xi)) = J_l(xi) J_l(-xi)^-1
        assert np.abs(O.adj(O.exp(xi)) - J @ np.linalg.inv(O.left_jacobian(-xi))).max() < 1e-11 * np.abs(J).max() ** 2
