"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake in the oracle: a dropped term, a wrong
sign, a wrong branch boundary, a transposed operand, a wrong prefactor.
None of them compare the oracle with a retyped copy of its own formula.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_bead.txt")


def _num(tok):
    return float(Fraction(tok))


def _golden_cases():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "case":
            cur = {"name": vals[0]}
            cases.append(cur)
        else:
            cur[key] = np.array([_num(v) for v in vals])
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_two_bead_golden(case):
    a, s = 1.0, 6 * math.pi
    pos = np.array([case["R"], [0.0, 0.0, 0.0]])
    f = np.array([case["F1"], case["F2"]])
    u = oracle.rpy_direct(pos, f, a, s)
    np.testing.assert_allclose(u[0], case["u1"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[1], case["u2"], rtol=0, atol=1e-14)


def dense_matrix(pos, a, s):
    """The 3N x 3N tensor, column by column, from the oracle matvec."""
    n = pos.shape[0]
    D = np.zeros((3 * n, 3 * n))
    for c in range(3 * n):
        e = np.zeros((n, 3))
        e[c // 3, c % 3] = 1.0
        D[:, c] = oracle.rpy_direct(pos, e, a, s, threads=1).ravel()
    return D


def test_symmetry_and_reciprocity():
    rng = np.random.default_rng(1)
    pos = rng.random((40, 3)) * 0.3          # many overlapping pairs at a = 0.03
    D = dense_matrix(pos, 0.03, 1.7)
    assert np.abs(D - D.T).max() < 1e-14 * np.abs(D).max()
    # each 3x3 block is itself symmetric (D_ij = D_ij^T)
    blk = D.reshape(40, 3, 40, 3)
    assert np.abs(blk - blk.transpose(0, 3, 2, 1)).max() < 1e-14 * np.abs(D).max()


@pytest.mark.parametrize("kind", ["uniform", "overlapping", "coincident"])
def test_positive_definite(kind):
    """Sec. 1: the RPY tensor is positive definite (Cholesky of the dense matrix)."""
    rng = np.random.default_rng(7)
    n = 200 if kind != "coincident" else 60
    if kind == "uniform":
        pos, a = rng.random((n, 3)), 0.02
    elif kind == "overlapping":
        pos, a = rng.random((n, 3)) * 0.5, 0.08      # mean spacing < 2a
    else:
        pos, a = rng.random((n, 3)), 0.05
        pos[1::2] = pos[0::2] + 1e-3 * rng.standard_normal((n // 2, 3))
    D = dense_matrix(pos, a, 6 * math.pi * a)
    np.linalg.cholesky(D)
    assert np.linalg.eigvalsh(D).min() > 0


def _block(r_vec, a, s):
    pos = np.array([r_vec, [0.0, 0.0, 0.0]])
    cols = []
    for k in range(3):
        f = np.zeros((2, 3))
        f[1, k] = 1.0
        cols.append(oracle.rpy_direct(pos, f, a, s, threads=1)[0])
    return np.array(cols).T


def test_continuity_at_contact():
    """Both branches meet at r = 2a (the printed overlap form would jump)."""
    a, s = 0.37, 2.3
    d = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    lo = _block(d * 2 * a * (1 - 1e-10), a, s)
    hi = _block(d * 2 * a * (1 + 1e-10), a, s)
    assert np.abs(lo - hi).max() < 1e-9 * np.abs(hi).max()
    # slope check: the overlap branch approaches from below smoothly
    lo2 = _block(d * 2 * a * (1 - 1e-4), a, s)
    assert np.abs(lo2 - hi).max() < 1e-3 * np.abs(hi).max()


def test_r_to_zero_limit():
    a, s = 0.5, 1.0
    self_c = s / (6 * math.pi * a)
    b0 = _block([0.0, 0.0, 0.0], a, s)
    np.testing.assert_allclose(b0, self_c * np.eye(3), rtol=1e-15, atol=0)
    b1 = _block([1e-9, 2e-9, -1e-9], a, s)
    np.testing.assert_allclose(b1, self_c * np.eye(3), rtol=0, atol=1e-8 * self_c)


def test_single_bead_is_self_term():
    f = np.array([[0.3, -1.2, 2.0]])
    u = oracle.rpy_direct(np.array([[0.1, 0.2, 0.3]]), f, 0.25, 4.0)
    np.testing.assert_allclose(u, 4.0 / (6 * math.pi * 0.25) * f, rtol=1e-15)


def test_linearity():
    rng = np.random.default_rng(3)
    pos = rng.random((50, 3))
    f1, f2 = rng.standard_normal((2, 50, 3))
    a = 0.05
    u1 = oracle.rpy_direct(pos, f1, a, 1.0)
    u2 = oracle.rpy_direct(pos, f2, a, 1.0)
    u12 = oracle.rpy_direct(pos, 2.0 * f1 - 3.0 * f2, a, 1.0)
    np.testing.assert_allclose(u12, 2 * u1 - 3 * u2, rtol=1e-12, atol=1e-12)
    u1s = oracle.rpy_direct(pos, f1, a, 5.0)
    np.testing.assert_allclose(u1s, 5 * u1, rtol=1e-13)


def test_oseen_limit():
    """a -> 0 at fixed kT/eta: the pair blocks tend to the Oseen tensor
    (1/(8 pi r))(I + RR/r^2); the a^2/r^2 term vanishes."""
    rng = np.random.default_rng(5)
    pos = rng.random((20, 3))
    f = rng.standard_normal((20, 3))
    a = 1e-7
    u = oracle.rpy_direct(pos, f, a, 1.0) - f / (6 * math.pi * a)
    ref = np.zeros_like(u)
    for i in range(20):
        for j in range(20):
            if i != j:
                R = pos[i] - pos[j]
                r = np.linalg.norm(R)
                ref[i] += (np.eye(3) + np.outer(R, R) / r ** 2) @ f[j] / (8 * math.pi * r)
    np.testing.assert_allclose(u, ref, rtol=1e-9, atol=1e-9)


def test_rotation_and_translation():
    rng = np.random.default_rng(11)
    pos = rng.random((60, 3)) * 0.4
    f = rng.standard_normal((60, 3))
    a = 0.03
    u = oracle.rpy_direct(pos, f, a, 1.0)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    uq = oracle.rpy_direct(pos @ Q.T, f @ Q.T, a, 1.0)
    np.testing.assert_allclose(uq, u @ Q.T, rtol=1e-11, atol=1e-11)
    ut = oracle.rpy_direct(pos + np.array([1e3, -1e3, 1e3]), f, a, 1.0)
    np.testing.assert_allclose(ut, u, rtol=1e-9, atol=1e-9)


def test_target_subset_matches_full():
    rng = np.random.default_rng(2)
    pos = rng.random((300, 3))
    f = rng.standard_normal((300, 3))
    full = oracle.rpy_direct(pos, f, 0.01, 1.0)
    idx = np.array([5, 17, 299, 0, 150])
    part = oracle.rpy_direct(pos, f, 0.01, 1.0, targets=idx)
    np.testing.assert_array_equal(part, full[idx])
    # bitwise independent of the thread count
    one = oracle.rpy_direct(pos, f, 0.01, 1.0, threads=1)
    np.testing.assert_array_equal(one, full)


# ---------------------------------------------------------------- Laplace split

def _far_config(rng, n, a, min_sep):
    """Random beads with every pair at least min_sep apart (by rejection)."""
    pts = []
    while len(pts) < n:
        p = rng.random(3) * 0.2
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts)


def test_laplace_single_charge_closed_form():
    y = np.array([[0.2, -0.1, 0.4]])
    x = np.array([[1.0, 0.5, -0.3]])
    phi, g, H = oracle.laplace_direct(y, np.array([2.5]), x)
    R = x[0] - y[0]
    r = np.linalg.norm(R)
    assert abs(phi[0, 0] - 2.5 / r) < 1e-15
    np.testing.assert_allclose(g[0, 0], -2.5 * R / r ** 3, rtol=1e-14)
    np.testing.assert_allclose(H[0, 0], 2.5 * (3 * np.outer(R, R) / r ** 5 - np.eye(3) / r ** 3), rtol=1e-13)


def test_laplace_derivatives_by_finite_differences():
    rng = np.random.default_rng(4)
    src = rng.random((30, 3))
    q = rng.standard_normal((30, 2))
    x0 = np.array([[1.7, 1.3, 1.9]])
    phi, g, H = oracle.laplace_direct(src, q, x0)
    h = 1e-5
    for k in range(3):
        e = np.zeros((1, 3))
        e[0, k] = h
        pp, gp, _ = oracle.laplace_direct(src, q, x0 + e)
        pm, gm, _ = oracle.laplace_direct(src, q, x0 - e)
        np.testing.assert_allclose((pp - pm) / (2 * h), g[:, :, k], rtol=1e-8)
        np.testing.assert_allclose((gp - gm) / (2 * h), H[:, :, :, k], rtol=1e-7, atol=1e-9)
    # harmonic: trace of the Hessian vanishes (Sec. 2, nabla_- nabla_+ = -nabla_0 nabla_0)
    assert np.abs(np.trace(H[0], axis1=1, axis2=2)).max() < 1e-12 * np.abs(H).max()


@pytest.mark.parametrize("origin", [(0.0, 0.0, 0.0), (0.1, 0.1, 0.1), (1e3, -1e3, 1e3)])
def test_far_split_equals_tensor(origin):
    """Eq. (2.8) with -C2 grad L_C reproduces the far branch of the tensor.
    Sources sit at 2a..8a from the targets, where the a^2/r^2 term matters."""
    rng = np.random.default_rng(9)
    a = 0.01
    pos = _far_config(rng, 40, a, 2.0 * a)
    f = rng.standard_normal((40, 3))
    s = 1.3
    u_t = oracle.rpy_direct(pos, f, a, s) - s / (6 * math.pi * a) * f
    u_s = oracle.rpy_far_split(pos, f, pos, a, s, origin=origin)
    tol = 1e-11 if origin[0] < 1 else 1e-7
    assert oracle.rel_l2(u_s, u_t) < tol


def test_far_split_printed_sign_is_wrong():
    """The printed +C2 grad L_C (Eq. 2.8) disagrees with the tensor."""
    rng = np.random.default_rng(9)
    a = 0.01
    pos = _far_config(rng, 40, a, 2.0 * a)
    f = rng.standard_normal((40, 3))
    u_t = oracle.rpy_direct(pos, f, a, 1.0) - 1.0 / (6 * math.pi * a) * f
    u_p = oracle.rpy_far_split(pos, f, pos, a, 1.0, dipole_sign=+1.0)
    assert oracle.rel_l2(u_p, u_t) > 1e-3


# ---------------------------------------------------------------- tree keys

def test_morton_hand_values():
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.5, 0.0, 0.0],
                    [0.0, 0.5, 0.0], [0.0, 0.0, 0.5], [0.25, 0.75, 0.0]])
    keys, cube = oracle.morton_keys(pos)
    np.testing.assert_array_equal(cube, [0.5, 0.5, 0.5, 1.0])
    assert int(keys[0]) == 0
    assert int(keys[1]) == (1 << 63) - 1          # clamped to 2^21 - 1 on every axis
    assert int(keys[2]) == 1 << 60                 # x bit 20
    assert int(keys[3]) == 1 << 61                 # y bit 20
    assert int(keys[4]) == 1 << 62                 # z bit 20
    # x = 0.25 -> q = 2^19 (bit 19 of x -> key bit 57); y = 0.75 -> bits 20, 19 of y
    assert int(keys[5]) == (1 << 57) | (1 << 61) | (1 << 58)


def test_morton_degenerate_and_anisotropic():
    keys, cube = oracle.morton_keys(np.array([[0.3, 0.3, 0.3]] * 4))
    assert np.all(keys == 0) and cube[3] == 0.0
    # the cube side is the largest extent; other axes are centred
    keys, cube = oracle.morton_keys(np.array([[0.0, 0.0, 0.0], [2.0, 0.5, 0.0]]))
    np.testing.assert_array_equal(cube, [1.0, 0.25, 0.0, 2.0])
    # y: (0.5 - (0.25 - 1)) / 2 = 0.625 -> q_y = 0.625 * 2^21 = bits 20 and 18
    # z: (0 - (0 - 1)) / 2 = 0.5 -> bit 20
    qy = int(0.625 * 2 ** 21)
    assert qy == (1 << 20) | (1 << 18)
    expect = (((1 << 21) - 1, qy, 1 << 20))
    key = 0
    for b in range(20, -1, -1):
        key = (key << 3) | (((expect[2] >> b) & 1) << 2) | (((expect[1] >> b) & 1) << 1) | ((expect[0] >> b) & 1)
    assert int(keys[1]) == key


def test_stable_sort_brute_force():
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 20, size=3000).astype(np.uint64)
    perm = oracle.stable_sort(keys)
    assert sorted(perm.tolist()) == list(range(3000))
    ks = keys[perm]
    assert np.all(ks[1:] >= ks[:-1])
    same = ks[1:] == ks[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])           # ties keep index order
    ref = sorted(range(3000), key=lambda i: (int(keys[i]), i))
    np.testing.assert_array_equal(perm, ref)


def test_rel_l2():
    assert oracle.rel_l2([[3.0, 4.0, 0.0]], [[0.0, 0.0, 5.0]]) == pytest.approx(math.sqrt(50) / 5)
    assert oracle.rel_l2([[1.0, 1.0, 1.0]], [[1.0, 1.0, 1.0]]) == 0.0
