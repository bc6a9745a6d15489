"""CPU check of the structure the fine-level CUDA kernel relies on: in the
Walsh-Hadamard basis of the corner signs, the unit hex8 stiffness is block
diagonal over the eight reflection-parity classes of (monomial, component),
and the constant monomial (rigid translation) carries no energy."""

import itertools

import numpy as np
import pytest

from oracle import fem


def _mono(sigma, c):
    return ((sigma & 1) ^ (c == 0)) | ((((sigma >> 1) & 1) ^ (c == 1)) << 1) | ((((sigma >> 2) & 1) ^ (c == 2)) << 2)


@pytest.mark.parametrize("nu", [0.3, 0.2, 0.45])
def test_stiffness_block_diagonal_in_parity_classes(nu):
    Ke = fem.element_stiffness(nu)
    s = 2 * fem.LOCAL_NODES - 1                       # corner signs
    H = np.zeros((8, 8))
    for m in range(8):
        for a in range(8):
            H[m, a] = np.prod([s[a, k] for k in range(3) if (m >> k) & 1])
    H3 = np.kron(H, np.eye(3))                          # rows (m, c)
    G = H3 @ Ke @ H3.T / 64
    cls = np.zeros(24, dtype=int)
    for m, c in itertools.product(range(8), range(3)):
        cls[3 * m + c] = ((m & 1) ^ (c == 0)) | ((((m >> 1) & 1) ^ (c == 1)) << 1) | ((((m >> 2) & 1) ^ (c == 2)) << 2)
    same = cls[:, None] == cls[None, :]
    assert np.max(np.abs(G[~same])) < 1e-14
    assert np.max(np.abs(G[0:3, :])) < 1e-14 and np.max(np.abs(G[:, 0:3])) < 1e-14
    # each class holds exactly one (monomial, component) pair per component
    for sig in range(8):
        members = sorted(3 * _mono(sig, c) + c for c in range(3))
        assert sorted(np.flatnonzero(cls == sig)) == members
    # and the factorisation reproduces K_e
    assert np.max(np.abs(H3.T @ G @ H3 - Ke)) < 1e-14


def _blocks(nu):
    """G as [class][row][column] (rows and columns: the class's components)."""
    Ke = fem.element_stiffness(nu)
    s = 2 * fem.LOCAL_NODES - 1
    H = np.zeros((8, 8))
    for m in range(8):
        for a in range(8):
            H[m, a] = np.prod([s[a, k] for k in range(3) if (m >> k) & 1])
    G = np.kron(H, np.eye(3)) @ Ke @ np.kron(H, np.eye(3)).T / 64
    return np.array([[[G[3 * _mono(sg, i) + i, 3 * _mono(sg, j) + j] for j in range(3)] for i in range(3)]
                     for sg in range(8)]), G


def _factored(vals, u):
    """w = G u in the factored form of the kernels (u, w: [mode 0..7][component])."""
    a, b, a7, b7, p, q, c, d = vals
    w = np.zeros((8, 3))
    t = b * (u[1, 0] + u[2, 1] + u[4, 2])
    w[1, 0], w[2, 1], w[4, 2] = (a - b) * u[1, 0] + t, (a - b) * u[2, 1] + t, (a - b) * u[4, 2] + t
    t = b7 * (u[6, 0] + u[5, 1] + u[3, 2])
    w[6, 0], w[5, 1], w[3, 2] = (a7 - b7) * u[6, 0] + t, (a7 - b7) * u[5, 1] + t, (a7 - b7) * u[3, 2] + t
    w[3, 1], w[5, 2] = p * u[3, 1] + q * u[5, 2], q * u[3, 1] + p * u[5, 2]
    w[3, 0], w[6, 2] = p * u[3, 0] + q * u[6, 2], q * u[3, 0] + p * u[6, 2]
    w[5, 0], w[6, 1] = p * u[5, 0] + q * u[6, 1], q * u[5, 0] + p * u[6, 1]
    w[2, 0] = w[1, 1] = c * (u[2, 0] + u[1, 1])
    w[7, 2] = d * u[7, 2]
    w[4, 0] = w[1, 2] = c * (u[4, 0] + u[1, 2])
    w[7, 1] = d * u[7, 1]
    w[4, 1] = w[2, 2] = c * (u[4, 1] + u[2, 2])
    w[7, 0] = d * u[7, 0]
    return w


@pytest.mark.parametrize("nu", [0.0, 0.1, 0.2, 0.3, 0.45, 0.49])
def test_parity_blocks_take_eight_values(nu):
    """The fine kernels apply G in a form reduced by the cube's symmetry: eight
    distinct values (a, b of class 0; a', b' of class 7; p, q of the 2x2 blocks
    of classes 1, 2, 4; c, d of classes 3, 5, 6) and 27 zeros, for any nu."""
    g, G = _blocks(nu)
    big = np.max(np.abs(g))
    a, b = g[0, 0, 0], g[0, 0, 1]
    a7, b7 = g[7, 0, 0], g[7, 0, 1]
    p, q = g[1, 1, 1], g[1, 1, 2]
    c, d = g[3, 0, 0], g[3, 2, 2]
    want = np.zeros((8, 3, 3))
    want[0] = b + (a - b) * np.eye(3)
    want[7] = b7 + (a7 - b7) * np.eye(3)
    for sg, (r0, r1) in ((1, (1, 2)), (2, (0, 2)), (4, (0, 1))):
        want[sg, r0, r0] = want[sg, r1, r1] = p
        want[sg, r0, r1] = want[sg, r1, r0] = q
    for sg, (r0, r1), rd in ((3, (0, 1), 2), (5, (0, 2), 1), (6, (1, 2), 0)):
        for i in (r0, r1):
            for j in (r0, r1):
                want[sg, i, j] = c
        want[sg, rd, rd] = d
    assert np.max(np.abs(g - want)) < 1e-13 * big
    assert np.count_nonzero(np.abs(want) > 0) == 45 or nu == 0.0
    # the factored contraction equals the dense one on random modes
    rng = np.random.default_rng(3)
    for _ in range(5):
        u = rng.standard_normal((8, 3))
        dense = (G @ u.reshape(24)).reshape(8, 3)
        got = _factored((a, b, a7, b7, p, q, c, d), u)
        assert np.max(np.abs(got[1:] - dense[1:])) < 1e-13 * big * np.max(np.abs(u))
        assert np.max(np.abs(dense[0])) < 1e-13 * big * np.max(np.abs(u))
