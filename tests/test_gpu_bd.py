"""GPU checks of the Brownian-dynamics consumers of the matvec, through the C ABI.

rpy_lanczos_sqrt against the square root of the dense 3N x 3N RPY matrix that
the oracle assembles column by column (small N, one leaf, so that the GPU
matvec is the exact direct sum); against invariants at FMM sizes
(|D^{1/2} z|^2 = z.D z and D^{1/2} D^{1/2} z = D z, with the oracle's D z);
and rpy_bd_step against its definition r + (dt/kT) D F + sqrt(2 dt) D^{1/2} xi.
"""
import numpy as np
import pytest

import oracle
import paper_1711_02976_gb300 as rp
import synth
from gpu_util import cuda_tensor

pytestmark = pytest.mark.gpu


def _dense_D(pos, a, s):
    n = len(pos)
    D = np.zeros((3 * n, 3 * n))
    for j in range(n):
        for c in range(3):
            f = np.zeros((n, 3))
            f[j, c] = 1.0
            D[:, 3 * j + c] = oracle.rpy_direct(pos, f, a, s).ravel()
    return D


def _sqrtm_psd(D):
    lam, Q = np.linalg.eigh(0.5 * (D + D.T))
    return (Q * np.sqrt(np.clip(lam, 0.0, None))) @ Q.T


def test_lanczos_matches_dense_square_root():
    rng = np.random.default_rng(7)
    sysm = synth.uniform_cube(40, seed=8, a=0.03)   # some pairs overlap (r < 2a)
    D = _dense_D(sysm.pos, sysm.a, sysm.s)
    R = _sqrtm_psd(D)
    assert np.allclose(R @ R, D, rtol=0, atol=1e-12 * np.abs(D).max())   # the reference itself
    z = rng.standard_normal((sysm.n, 3))
    t = rp.rpy_forest_build(cuda_tensor(sysm.pos), [0, sysm.n], [sysm.a], 6, leaf_cap=64)
    import torch
    Y = torch.empty((sysm.n, 3), dtype=torch.float64, device="cuda")
    steps, change = rp.rpy_lanczos_sqrt(t, cuda_tensor(z), sysm.s, Y, m_max=3 * sysm.n, tol=1e-12)
    y = Y.cpu().numpy().ravel()
    ref = R @ z.ravel()
    assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref), (steps, change)


def test_lanczos_forest_is_block_diagonal():
    rng = np.random.default_rng(9)
    A = synth.uniform_cube(25, seed=10, a=0.04)
    B = synth.uniform_cube(30, seed=11, a=0.02)
    pos = np.concatenate([A.pos, B.pos])
    z = rng.standard_normal((A.n + B.n, 3))
    t = rp.rpy_forest_build(cuda_tensor(pos), [0, A.n, A.n + B.n], [A.a, B.a], 6, leaf_cap=64)
    import torch
    Y = torch.empty((A.n + B.n, 3), dtype=torch.float64, device="cuda")
    rp.rpy_lanczos_sqrt(t, cuda_tensor(z), [A.s, 3.0 * B.s], Y, m_max=3 * (A.n + B.n), tol=1e-12)
    y = Y.cpu().numpy()
    ra = _sqrtm_psd(_dense_D(A.pos, A.a, A.s)) @ z[:A.n].ravel()
    rb = _sqrtm_psd(_dense_D(B.pos, B.a, 3.0 * B.s)) @ z[A.n:].ravel()
    ref = np.concatenate([ra, rb])
    assert np.linalg.norm(y.ravel() - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [rp.RPY_FP64, rp.RPY_FP32])
def test_lanczos_invariants_at_fmm_size(precision):
    rng = np.random.default_rng(12)
    sysm = synth.sphere_plus_cube(20000, seed=13, a=5e-4)
    z = rng.standard_normal((sysm.n, 3))
    t = rp.rpy_forest_build(cuda_tensor(sysm.pos), [0, sysm.n], [sysm.a], 6, precision=precision)
    import torch
    Y = torch.empty((sysm.n, 3), dtype=torch.float64, device="cuda")
    Y2 = torch.empty_like(Y)
    # the FMM matvec carries a ~1e-7 relative error, so the Lanczos steps stop changing y
    # at about that level: ask for 1e-6
    steps, change = rp.rpy_lanczos_sqrt(t, cuda_tensor(z), sysm.s, Y, m_max=100, tol=1e-6)
    assert steps < 100 and change <= 1e-6, (steps, change)
    rp.rpy_lanczos_sqrt(t, Y, sysm.s, Y2, m_max=100, tol=1e-6)
    y, y2 = Y.cpu().numpy(), Y2.cpu().numpy()
    Dz = oracle.rpy_direct(sysm.pos, z, sysm.a, sysm.s)
    zDz = float(np.sum(z * Dz))
    assert abs(float(np.sum(y * y)) - zDz) <= 1e-5 * zDz
    assert np.linalg.norm(y2 - Dz) <= 1e-5 * np.linalg.norm(Dz)


def test_bd_step_follows_its_definition():
    rng = np.random.default_rng(14)
    sysm = synth.uniform_cube(40, seed=15, a=0.03)
    f = rng.standard_normal((sysm.n, 3))
    xi = rng.standard_normal((sysm.n, 3))
    kT, eta, dt = 2.5, 0.7, 1e-3
    s = kT / eta
    P = cuda_tensor(sysm.pos)
    t = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], 6, leaf_cap=64)
    import torch
    disp = torch.empty_like(P)
    rp.rpy_bd_step(t, P, cuda_tensor(f), cuda_tensor(xi), kT, eta, dt, m_max=3 * sysm.n, tol=1e-12, disp=disp)
    D = _dense_D(sysm.pos, sysm.a, s)
    ref = (dt / kT) * (D @ f.ravel()) + np.sqrt(2 * dt) * (_sqrtm_psd(D) @ xi.ravel())
    d = disp.cpu().numpy().ravel()
    assert np.linalg.norm(d - ref) <= 1e-9 * np.linalg.norm(ref)
    new = P.cpu().numpy()
    assert np.max(np.abs(new - (sysm.pos + d.reshape(-1, 3)))) <= 1e-15
    # the tree now describes the new positions
    U = torch.empty_like(P)
    rp.rpy_forest_matvec(t, cuda_tensor(f), [s], U)
    rp.rpy_tree_sync(t)
    uref = oracle.rpy_direct(new, f, sysm.a, s)
    assert np.max(np.abs(U.cpu().numpy() - uref)) <= 1e-12 * np.max(np.abs(uref))
