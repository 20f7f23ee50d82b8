"""Host-side logic of the library, checked on the CPU (no GPU needed):
exported symbols, argument validation without a device, and the FMM operator
tables against independent test-side harmonics and direct 1/r sums."""
import math
import os
import re

import numpy as np
import pytest

import paper_1711_02976_gb300 as rp
from harmonics_ref import as_real, eval_real, from_real, irregular, ncoef, p2l, p2m, regular, tri

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rpyfmm.h")


def test_library_exports_every_declared_symbol():
    lib = rp.load()
    names = re.findall(r"^\s*(?:int64_t|int|void|const char \*)\s*\*?\s*(rpy_\w+)\s*\(", open(HEADER).read(), re.M)
    assert len(names) >= 18
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) == set(rp.EXPORTED_SYMBOLS)
    assert rp.rpy_version() >= 100


def test_strerror_and_validation_without_device():
    assert rp.rpy_strerror(0) == "success"
    assert "digits" in rp.rpy_strerror(-2)
    lib = rp.load()
    import ctypes
    out = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    # argument errors are reported before any device access
    assert lib.rpy_tree_build(fake, 0, 0.1, 3, 0, 0, None, ctypes.byref(out)) == -1
    assert lib.rpy_tree_build(fake, 10, -1.0, 3, 0, 0, None, ctypes.byref(out)) == -1
    assert lib.rpy_tree_build(fake, 10, 0.1, 4, 0, 0, None, ctypes.byref(out)) == -2
    assert lib.rpy_tree_build(None, 10, 0.1, 3, 0, 0, None, ctypes.byref(out)) == -1
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        # valid arguments, no device: fails loudly, never computes on the CPU
        assert lib.rpy_tree_build(fake, 10, 0.1, 3, 0, 0, None, ctypes.byref(out)) == -8
        assert out.value is None
    assert lib.rpy_matvec(None, fake, 1.0, fake, None) == -1
    assert rp.rpy_tree_footprint(10 ** 6, 6) > 10 ** 6
    # sampled direct sum and autotuner: argument checks, then no device
    off = np.array([0, 10], dtype=np.int64)
    bad_off = np.array([0, 0], dtype=np.int64)
    av, sv = np.array([0.1]), np.array([1.0])
    tg = np.array([0, 3], dtype=np.int64)
    u = np.zeros((2, 3))
    res = rp.AutotuneResult()
    assert lib.rpy_direct_sampled(fake, bad_off.ctypes.data, 1, av.ctypes.data, fake, sv.ctypes.data,
                                  tg.ctypes.data, 2, u.ctypes.data, None) == -1
    assert lib.rpy_autotune(fake, off.ctypes.data, 1, av.ctypes.data, fake, sv.ctypes.data, 5, 0, None,
                            ctypes.byref(res), None) == -2
    assert lib.rpy_autotune(fake, off.ctypes.data, 1, av.ctypes.data, fake, sv.ctypes.data, 3, 0, None,
                            None, None) == -1
    # 9 digits: FP64 only
    assert lib.rpy_autotune(fake, off.ctypes.data, 1, av.ctypes.data, fake, sv.ctypes.data, 9, 1, None,
                            ctypes.byref(res), None) == -2
    assert rp.rpy_tree_footprint(10 ** 6, 9) > rp.rpy_tree_footprint(10 ** 6, 6)
    it, ch = ctypes.c_int(), ctypes.c_double()
    assert lib.rpy_lanczos_sqrt(None, fake, sv.ctypes.data, 10, 1e-8, fake, ctypes.byref(it), ctypes.byref(ch),
                                None) == -1
    assert lib.rpy_bd_step(None, fake, fake, fake, sv.ctypes.data, sv.ctypes.data, 1e-3, 10, 1e-8, None,
                           ctypes.byref(it), None) == -1
    if not has_gpu:
        assert lib.rpy_direct_sampled(fake, off.ctypes.data, 1, av.ctypes.data, fake, sv.ctypes.data,
                                      tg.ctypes.data, 2, u.ctypes.data, None) == -8
        assert lib.rpy_autotune(fake, off.ctypes.data, 1, av.ctypes.data, fake, sv.ctypes.data, 3, 0, None,
                                ctypes.byref(res), None) == -8


@pytest.mark.parametrize("p", [6, 10])
def test_m2m_table_matches_direct_multipoles(p):
    T = rp.rpy_debug_table(p, 3, 1)
    D = 2 * ncoef(p)
    T = T.reshape(8, D, D)
    rng = np.random.default_rng(p)
    for o in range(8):
        delta = np.array([0.25 if (o >> a) & 1 else -0.25 for a in range(3)])
        cp, hp = np.array([0.3, -0.2, 0.7]), 2.0
        cc, hc = cp + delta * hp, hp / 2
        src = cc + (rng.random((30, 3)) - 0.5) * hc
        q = rng.standard_normal(30)
        Mc = p2m(src, q, cc, hc, p)
        Mp = p2m(src, q, cp, hp, p)
        got = from_real(T[o].T @ as_real(Mc))
        assert np.abs(got - Mp).max() < 1e-12 * np.abs(Mp).max(), o


@pytest.mark.parametrize("p", [6, 10])
def test_l2l_table_matches_direct_locals(p):
    T = rp.rpy_debug_table(p, 3, 2)
    D = 2 * ncoef(p)
    T = T.reshape(8, D, D)
    rng = np.random.default_rng(p + 1)
    cp, hp = np.array([0.1, 0.2, -0.3]), 1.0
    src = cp + 6.0 * (rng.random((40, 3)) - 0.5)
    src = src[np.max(np.abs(src - cp), axis=1) > 2.0]
    q = rng.standard_normal(len(src))
    Lp = p2l(src, q, cp, hp, p)
    for o in range(8):
        delta = np.array([0.25 if (o >> a) & 1 else -0.25 for a in range(3)])
        cc, hc = cp + delta * hp, hp / 2
        Lc = from_real(T[o].T @ as_real(Lp))
        # both expansions give the same potential near the child centre
        x = cc + (rng.random((10, 3)) - 0.5) * hc
        phi_p = eval_real(Lp, regular((x - cp) / hp, p)) / hp
        phi_c = eval_real(Lc, regular((x - cc) / hc, p)) / hc
        assert np.abs(phi_p - phi_c).max() < 1e-11 * np.abs(phi_p).max(), o


FRAMES = {0: np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]]), 1: np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]])}


def _rot_apply(blocks, offs, p, f, c):
    """Apply the per-degree real rotation blocks of frame f to complex coefficients c."""
    out = np.zeros_like(c)
    L = int(offs[-1])
    for n in range(p + 1):
        B = 2 * (n + 1)
        R = blocks[f * L + int(offs[n]): f * L + int(offs[n]) + B * B].reshape(B, B)
        xr = as_real(c[tri(n, 0): tri(n, 0) + n + 1])
        out[tri(n, 0): tri(n, 0) + n + 1] = from_real(R @ xr)
    return out


@pytest.mark.parametrize("f", [0, 1])
def test_frame_rotations(f):
    p = 8
    fwd = rp.rpy_debug_table(p, 3, 3)
    bwd = rp.rpy_debug_table(p, 3, 4)
    offs = rp.rpy_debug_table(p, 3, 10)
    Q = FRAMES[f]
    rng = np.random.default_rng(3)
    src = rng.random((20, 3)) - 0.5
    q = rng.standard_normal(20)
    M = p2m(src, q, np.zeros(3), 1.0, p)
    Mf = _rot_apply(fwd, offs, p, f, M)
    Mref = p2m(src @ Q.T, q, np.zeros(3), 1.0, p)     # coordinates in the frame
    assert np.abs(Mf - Mref).max() < 1e-12
    # backward: a local expansion written in frame coordinates, mapped to world
    far = rng.random((15, 3)) * 2 + 3.0
    qf = rng.standard_normal(15)
    Lf = p2l(far @ Q.T, qf, np.zeros(3), 1.0, p)
    Lw = _rot_apply(bwd, offs, p, f, Lf)
    assert np.abs(Lw - p2l(far, qf, np.zeros(3), 1.0, p)).max() < 1e-12


def _quad(digits, p):
    q = rp.rpy_debug_table(p, digits, 11)
    s = int(q[0])
    lam, w, M = q[1::3][:s], q[2::3][:s], q[3::3][:s].astype(int)
    return s, lam, w, M


@pytest.mark.parametrize("digits,tol", [(3, 3.0e-4), (4, 4.0e-5), (5, 3.5e-6), (6, 4.5e-7), (9, 2.5e-10)])
def test_lambda_quadrature(digits, tol):
    from scipy.special import j0
    s, lam, w, M = _quad(digits, 10)
    assert np.all(M % 2 == 0) and np.all(np.diff(lam) > 0) and np.all(w > 0)
    z = np.linspace(1, 4, 41)[:, None]
    rho = np.linspace(0, 4 * math.sqrt(2), 57)[None, :]
    approx = sum(w[k] * np.exp(-lam[k] * z) * j0(lam[k] * rho) for k in range(s))
    err = np.abs(approx * np.sqrt(z ** 2 + rho ** 2) - 1).max()
    assert err < tol


# direction -> signed permutation (frame coordinates = P @ world)
PD = {0: np.eye(3), 1: np.diag([1, 1, -1]),
      2: np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]]), 3: np.array([[0, 1, 0], [0, 0, 1], [-1, 0, 0]]),
      4: np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]]), 5: np.array([[0, 0, 1], [1, 0, 0], [0, -1, 0]])}
# a V-list offset (target centre - source centre, box units) in each direction
OFFSETS = {0: (1, -2, 3), 1: (0, 1, -2), 2: (2, 1, -1), 3: (-3, 0, 1), 4: (3, 2, 0), 5: (-1, -3, 1)}


def _classify(D):
    if D[2] >= 2: return 0
    if D[2] <= -2: return 1
    if D[1] >= 2: return 4
    if D[1] <= -2: return 5
    if D[0] >= 2: return 2
    if D[0] <= -2: return 3
    return -1


def _plane_wave_chain(M, d, off, p, digits):
    """M (world, source box units) -> local expansion about the target centre, via the
    library's M2X / X2L tables and a directly computed diagonal shift."""
    nc = ncoef(p)
    s, lam, w, Mk = _quad(digits, p)
    pw = rp.rpy_debug_table(p, digits, 7).reshape(-1, 4)
    ek, ca, sa, wm = pw[:, 0].astype(int), pw[:, 1], pw[:, 2], pw[:, 3]
    c_m2x = rp.rpy_debug_table(p, digits, 5).reshape(s, nc)
    c_x2l = rp.rpy_debug_table(p, digits, 6).reshape(s, nc)
    fwd, bwd, offs = rp.rpy_debug_table(p, digits, 3), rp.rpy_debug_table(p, digits, 4), rp.rpy_debug_table(p, digits, 10)
    f = d // 2
    Mf = M if f == 0 else _rot_apply(fwd, offs, p, f - 1, M)
    nm = np.array([n + m for n in range(p + 1) for m in range(n + 1)])
    sgn = np.where(nm % 2 == 0, 1.0, -1.0)
    if d & 1:
        Mf = Mf * sgn
    A = c_m2x * Mf[None, :]                       # (s, nc)
    mm = np.array([m for n in range(p + 1) for m in range(n + 1)])
    Akm = np.zeros((s, p + 1), complex)
    for m in range(p + 1):
        Akm[:, m] = A[:, mm == m].sum(axis=1)
    alpha = np.arctan2(sa, ca)
    W = np.zeros(len(ek), complex)
    for e in range(len(ek)):
        k = ek[e]
        v = Akm[k, 0].real
        for m in range(1, p + 1):
            v = v + 2 * (1j ** m) * np.real(Akm[k, m] * np.exp(1j * m * alpha[e]))
        W[e] = wm[e] * v
    Dp = PD[d] @ np.asarray(off, float)
    lam_e = lam[ek]
    W = W * np.exp(-lam_e * Dp[2] + 1j * lam_e * (Dp[0] * ca + Dp[1] * sa))
    Lf = np.zeros(nc, complex)
    for k in range(s):
        sel = ek == k
        for n in range(p + 1):
            for m in range(n + 1):
                b = np.sum((W[sel] + (-1) ** m * np.conj(W[sel])) * np.exp(-1j * m * alpha[sel]))
                Lf[tri(n, m)] += (1j ** m) * c_x2l[k, tri(n, m)] * b
    if d & 1:
        Lf = Lf * sgn
    return Lf if f == 0 else _rot_apply(bwd, offs, p, f - 1, Lf)


@pytest.mark.parametrize("digits,p,tol", [(3, 10, 2e-3), (5, 16, 2e-5), (6, 20, 3e-6), (9, 24, 2e-10)])
@pytest.mark.parametrize("d", range(6))
def test_plane_wave_m2l_chain(d, digits, p, tol):
    off = np.array(OFFSETS[d], float)
    assert _classify(off) == d
    rng = np.random.default_rng(10 + d)
    src = rng.random((25, 3)) - 0.5
    q = rng.standard_normal(25)
    M = p2m(src, q, np.zeros(3), 1.0, p)
    L = _plane_wave_chain(M, d, off, p, digits)
    tgt = off + rng.random((30, 3)) - 0.5
    phi = eval_real(L, regular(tgt - off, p))
    ref = np.array([np.sum(q / np.linalg.norm(x - src, axis=1)) for x in tgt])
    assert np.sqrt(np.sum((phi - ref) ** 2) / np.sum(ref ** 2)) < tol


def test_shift_table_formula():
    p, digits = 8, 3
    s, lam, w, Mk = _quad(digits, p)
    pw = rp.rpy_debug_table(p, digits, 7).reshape(-1, 4)
    S = pw.shape[0]
    assert S == Mk.sum() // 2
    sh = rp.rpy_debug_table(p, digits, 8).reshape(216, S, 2)
    for off in (0, 77, 215):
        dx, dy, dz = off % 6 - 2.5, (off // 6) % 6 - 2.5, off // 36 - 2.5
        le = lam[pw[:, 0].astype(int)]
        ref = np.exp(-le * dz + 1j * le * (dx * pw[:, 1] + dy * pw[:, 2]))
        np.testing.assert_allclose(sh[off, :, 0] + 1j * sh[off, :, 1], ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("digits", [3, 6])
def test_per_axis_shift_factors_multiply_to_the_shift_table(digits):
    """The FP32 X2X forms each plane-wave shift from per-axis factors: their
    product must be the full shift e^{-lambda dz + i lambda (dx cos a + dy sin a)}."""
    p = 8
    pw = rp.rpy_debug_table(p, digits, 7).reshape(-1, 4)
    S = pw.shape[0]
    sh = rp.rpy_debug_table(p, digits, 8).reshape(216, S, 2)
    sz = rp.rpy_debug_table(p, digits, 16).reshape(6, S)
    sx = rp.rpy_debug_table(p, digits, 17).reshape(6, S, 2)
    sy = rp.rpy_debug_table(p, digits, 18).reshape(6, S, 2)
    cx, cy = sx[..., 0] + 1j * sx[..., 1], sy[..., 0] + 1j * sy[..., 1]
    for off in range(216):
        ix, iy, iz = off % 6, (off // 6) % 6, off // 36
        prod = sz[iz] * cx[ix] * cy[iy]
        np.testing.assert_allclose(prod, sh[off, :, 0] + 1j * sh[off, :, 1], rtol=1e-13, atol=1e-13)


def test_merge_and_shift_groups_cover_v_lists():
    """Every (child of a parent, child of a colleague) pair that is not adjacent
    is served by exactly one direction and one group; adjacent pairs by none."""
    g = rp.rpy_debug_table(6, 3, 9).astype(int)
    pos = 0
    served = {}
    for d in range(6):
        ng = g[pos]; pos += 1
        for _ in range(ng):
            mask, cnt = g[pos], g[pos + 1]; pos += 2
            for z in range(cnt):
                slot = g[pos + z] & 255
                for t in range(8):
                    if (mask >> t) & 1:
                        key = (slot, t)
                        assert key not in served
                        served[key] = d
            pos += cnt
        pos += 8
    for q in range(27):
        dq = np.array([q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1])
        for o in range(8):
            s2 = 4 * dq + np.array([1 if (o >> a) & 1 else -1 for a in range(3)])
            for t in range(8):
                t2 = np.array([1 if (t >> a) & 1 else -1 for a in range(3)])
                D = (t2 - s2) // 2
                d = _classify(D)
                if d < 0:
                    assert (q * 8 + o, t) not in served
                else:
                    assert served[(q * 8 + o, t)] == d


@pytest.mark.parametrize("p", [6, 12])
def test_rotation_m2m_l2l_equal_dense_operators(p):
    """Rotate to the child's shift axis, shift along z, rotate back: the same
    linear maps as the dense addition-theorem operators."""
    nc = ncoef(p)
    D = 2 * nc
    dense_m = rp.rpy_debug_table(p, 3, 1).reshape(8, D, D)
    dense_l = rp.rpy_debug_table(p, 3, 2).reshape(8, D, D)
    fwd, bwd = rp.rpy_debug_table(p, 3, 12), rp.rpy_debug_table(p, 3, 13)
    zm = rp.rpy_debug_table(p, 3, 14).reshape(nc, p + 1)
    zl = rp.rpy_debug_table(p, 3, 15).reshape(nc, p + 1)
    offs = rp.rpy_debug_table(p, 3, 10)
    L = int(offs[-1])
    rng = np.random.default_rng(p)
    x = rng.standard_normal(nc) + 1j * rng.standard_normal(nc)
    for n in range(p + 1):
        x[tri(n, 0)] = x[tri(n, 0)].real

    def zshift(z, y, lower):
        out = np.zeros_like(y)
        for n in range(p + 1):
            for m in range(n + 1):
                ks = range(m, n + 1) if lower else range(n, p + 1)
                out[tri(n, m)] = sum(z[tri(n, m), k] * y[tri(k, m)] for k in ks)
        return out

    for o in range(8):
        f = np.concatenate([fwd[o * L:(o + 1) * L], fwd[o * L:(o + 1) * L]])
        b = np.concatenate([bwd[o * L:(o + 1) * L], bwd[o * L:(o + 1) * L]])
        ym = _rot_apply(b, offs, p, 0, zshift(zm, _rot_apply(f, offs, p, 0, x), True))
        np.testing.assert_allclose(ym, from_real(dense_m[o].T @ as_real(x)), rtol=0, atol=1e-12 * np.abs(x).max())
        yl = _rot_apply(b, offs, p, 0, zshift(zl, _rot_apply(f, offs, p, 0, x), False))
        np.testing.assert_allclose(yl, from_real(dense_l[o].T @ as_real(x)), rtol=0, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("n", [0, 1, 3, 6])
def test_coordinate_times_harmonic_splits_by_kelvin_transform(n):
    """The identity behind the one-expansion-per-component evaluation (approach 2
    of Sec. 2): for a harmonic polynomial h of degree n and g = h / (2n + 1),
        x_k h(x) = H(x) + |x|^2 d_k g(x),   H(x) = -|x|^(2n+3) d_k[g^K](x),
    where g^K is g with its coefficients read in the irregular basis (the Kelvin
    transform g / |x|^(2n+1)), and H is harmonic.  Checked by central differences
    with the test-side harmonics."""
    rng = np.random.default_rng(100 + n)
    c = np.zeros(ncoef(n), dtype=complex)
    for m in range(n + 1):
        c[tri(n, m)] = rng.standard_normal() + (1j * rng.standard_normal() if m else 0)
    g = c / (2 * n + 1)
    h = lambda x: eval_real(c, regular(x, n))
    gr = lambda x: eval_real(g, regular(x, n))
    gk = lambda x: eval_real(g, irregular(x, n))
    x = rng.uniform(-0.6, 0.6, (20, 3))
    e = 1e-5
    I = np.eye(3)
    r = np.linalg.norm(x, axis=1)
    for k in range(3):
        dg = (gr(x + e * I[k]) - gr(x - e * I[k])) / (2 * e)
        dgk = (gk(x + e * I[k]) - gk(x - e * I[k])) / (2 * e)
        H = -r ** (2 * n + 3) * dgk
        lhs = x[:, k] * h(x)
        assert np.max(np.abs(lhs - (H + r ** 2 * dg))) <= 1e-8 * max(1.0, np.max(np.abs(lhs)))
        # H is harmonic: its Laplacian by second differences vanishes
        Hf = lambda y: -np.linalg.norm(y, axis=1) ** (2 * n + 3) * (
            gk(y + e * I[k]) - gk(y - e * I[k])) / (2 * e)
        E = 1e-3
        lap = sum(Hf(x + E * I[a]) - 2 * Hf(x) + Hf(x - E * I[a]) for a in range(3)) / E ** 2
        assert np.max(np.abs(lap)) <= 1e-3 * max(1.0, np.max(np.abs(H)))
