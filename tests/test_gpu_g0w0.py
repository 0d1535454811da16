"""Plain G0W0 QP equation on the GPU (through the C ABI) against the FP64 oracle.

Eq. quasiparticle_equation with Sigma^c evaluated at eps itself has, for core levels, several
solutions (Sec. "Satellites in the G0W0 approximation"). The library solves it by the secant from
eps_n (qp_mode "g0w0") and lists every solution on a grid with its renormalisation factor Z
(gwc_g0w0_solutions). Tolerances: FP64 path 1e-8 Ha for the QP energy; bf16x3 the QP gate 1e-3 eV;
the grid scan is exact arithmetic on its input, so on the same Sigma array it matches the oracle's
scan to rounding, and on the FP64 GPU Sigma (1e-8 Ha from the oracle's) to 1e-6 Ha in position.
"""
import numpy as np
import pytest

from oracle import gwc_oracle as G
from paper_2412_17132_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EV = synth.HARTREE_EV


@pytest.fixture(scope="module")
def gwc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17132_gb300 import gwc as g

    g.lib()
    return g


@pytest.fixture(scope="module")
def mol():
    return synth.small(n_states=28, n_occ=6, n_core=2, n_aux=48, seed=21)


@pytest.fixture(scope="module")
def ref(mol):
    s = G.System.from_molecule(mol)
    eqp, dh, it = s.qp_solve(mode="g0w0")
    return s, eqp, dh


@pytest.mark.parametrize("prec,tol_ha", [("fp64", 1e-8), ("bf16x3", 1e-3 / EV)])
def test_g0w0_qp_matches_oracle(gwc, mol, ref, prec, tol_ha):
    s, eqp_ref, dh_ref = ref
    ctx = gwc.Context.from_molecule(mol, prec=prec, qp_mode="g0w0")
    e, dh, it = ctx.qp_solve()
    ctx.sync()
    for c in range(mol.n_core):
        assert abs(float(e[c]) - eqp_ref[c]) < tol_ha, (c, float(e[c]), eqp_ref[c])
        assert abs(float(dh[c]) - dh_ref[c]) < tol_ha


def _grid(mol, eqp):
    pts = [float(mol.eps[n]) for n in mol.core_idx] + [float(e) for e in eqp]
    return np.linspace(min(pts) - 1.0, max(pts) + 0.5, 401)


def test_g0w0_solutions_on_oracle_sigma_match_oracle_scan(gwc, mol, ref):
    """Same Sigma array on both sides: the device scan reproduces the oracle's roots and Z."""
    s = ref[0]
    grid = _grid(mol, ref[1])
    sig, _ = s.sigma_c_grid(grid)
    ctx = gwc.Context.from_molecule(mol, prec="fp64")
    sig_dev = torch.as_tensor(np.stack([sig.real, sig.imag], axis=-1), device="cuda").contiguous()
    roots, cnt = ctx.g0w0_solutions(torch.as_tensor(grid, device="cuda"), sig_dev)
    ctx.sync()
    sx, vxc = s.sigma_x(), s.v_xc()
    for c, n in enumerate(mol.core_idx):
        exp = G.g0w0_graphical_solutions(grid, sig[c], float(mol.eps[n]), sx[c], vxc[c])
        assert int(cnt[c]) == len(exp)
        got = roots[c, : len(exp)].cpu().numpy()
        for (x, z), (gx, gz) in zip(exp, got):
            assert abs(gx - x) < 1e-12 * max(1.0, abs(x))
            assert abs(gz - z) < 1e-9 * max(1.0, abs(z))


def test_g0w0_solutions_from_gpu_sigma_match_oracle(gwc, mol, ref):
    """End to end: FP64 GPU Sigma on the grid, device scan, against the oracle; at least one
    solution with 0 < Z < 1 per core, and the secant solution is within a grid step of one."""
    s, eqp_ref, _ = ref
    grid = _grid(mol, eqp_ref)
    ctx = gwc.Context.from_molecule(mol, prec="fp64")
    sig_dev, _, _ = ctx.sigma_core(grid)
    roots, cnt = ctx.g0w0_solutions(torch.as_tensor(grid, device="cuda"), sig_dev)
    ctx.sync()
    sig, _ = s.sigma_c_grid(grid)
    sx, vxc = s.sigma_x(), s.v_xc()
    step = grid[1] - grid[0]
    for c, n in enumerate(mol.core_idx):
        exp = G.g0w0_graphical_solutions(grid, sig[c], float(mol.eps[n]), sx[c], vxc[c])
        assert int(cnt[c]) == len(exp)
        got = roots[c, : len(exp)].cpu().numpy()
        for (x, z), (gx, gz) in zip(exp, got):
            assert abs(gx - x) < 1e-6
            assert abs(gz - z) < 1e-4 * max(1.0, abs(z))
        assert any(0 < z < 1 and abs(x - eqp_ref[c]) < step for x, z in exp)
