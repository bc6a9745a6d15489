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
