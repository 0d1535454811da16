"""Device-side failure statuses reach the host through gwc_sync, and the context stays usable.

No test here faults, traps or hangs the GPU: a bounded wait runs out because the context's wait
bound (gwc_options.wait_us) is set far below the time a tensor-core kernel's pipeline stages take,
so the kernel stops, drains what it issued, frees its tensor memory and returns; a QP iteration
stops at its iteration limit.
"""
import numpy as np
import pytest

from oracle import gwc_oracle as G
from paper_2412_17132_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17132_gb300 import gwc as g

    g.lib()
    return g


def test_exhausted_wait_reports_timeout_and_context_stays_usable(gwc):
    mol = synth.benzene()
    z = torch.tensor([[0.0, 0.7], [0.31, 1e-3], [9.9, 1e-3]], dtype=torch.float64, device="cuda")
    short = gwc.Context.from_molecule(mol, prec="bf16x3", wait_us=1)
    short.build_chi0(z)
    assert short.sync_status() == 6  # GWC_ERR_TIMEOUT
    assert short.sync_status() == 0  # the status word was cleared by the first sync
    # the same kernels with the default bound on a fresh context, and the GPU still answers
    ref_ctx = gwc.Context.from_molecule(mol, prec="bf16x3")
    out = ref_ctx.build_chi0(z)
    ref_ctx.sync()
    delta = G.transition_energies(mol.eps, mol.n_occ)
    ref = G.chi0(mol.o_ov, delta, complex(0.31, 1e-3))
    got = out[1].cpu().numpy()
    assert np.max(np.abs(got[..., 0] + 1j * got[..., 1] - ref)) <= 2e-5 * np.max(np.abs(ref))
    short.close()
    ref_ctx.close()


def test_qp_iteration_limit_reports_not_converged(gwc):
    mol = synth.tiny()
    ctx = gwc.Context.from_molecule(mol, prec="fp64", max_qp_iter=2, qp_mode="secant")
    with pytest.raises(gwc.GwcError) as e:
        ctx.qp_solve()
        ctx.sync()
    assert e.value.status == 5  # GWC_ERR_NOT_CONVERGED
    ok = gwc.Context.from_molecule(mol, prec="fp64")
    eqp, _, it = ok.qp_solve()
    ok.sync()
    assert int(it[0]) > 2
    ref, _, _ = G.System.from_molecule(mol).qp_solve()
    assert abs(float(eqp[0]) - ref[0]) < 1e-9


def test_chi0_builds_counted_only_when_done(gwc):
    """QP rounds launch every (core, occupied state) pair and skip converged ones; the stats count
    only the builds done: in the Hedin mode one round, i.e. the pairs with a residue at eps_n."""
    mol = synth.small(n_states=30, n_occ=6, n_core=3, n_aux=40, seed=31, n_omega=15)
    ctx = gwc.Context.from_molecule(mol, prec="bf16x3", qp_mode="hedin")
    ctx.qp_solve()
    ctx.sync()
    st = ctx.stats()
    eps_f = G.fermi_level(mol.eps, mol.n_occ)
    pairs = sum(1 for c in mol.core_idx for m in range(mol.n_occ)
                if G.residue_prefactor(mol.eps[m], float(mol.eps[c]), eps_f) != 0.0)
    table = mol.n_im + 1
    assert st["chi0_builds"] == table + pairs
    per = mol.n_aux * (mol.n_aux + 1.0) * mol.n_occ * (mol.n_states - mol.n_occ)
    assert abs(st["chi0_flop"] - per * (table + 2 * pairs)) <= 1e-9 * st["chi0_flop"]
