"""evGW0 through the C ABI (Sec. "GW for core-levels: beyond G0W0", Eq. ev_sigma_spectral) against the
FP64 oracle: every state of a 10-state system is a core, the QP energies of every state go back into
G, W keeps the RPA excitations of the input energies. Also the G-energy replacement of gwc_sigma_core
on its own, and the rejection of a virtual core by the paths that need occupied cores."""
import numpy as np
import pytest

from oracle import gwc_oracle as G
from paper_2412_17132_gb300 import synth
from test_oracle_pins import _all_state_system

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


def _ctx(gwc, s, prec):
    return gwc.Context(s.eps, s.n_occ, np.arange(s.n_states), s.o_ov, s.o_core, prec=prec, eta=s.eta, n_im=s.n_im,
                       xi0=s.xi0)


@pytest.mark.parametrize("prec,tol_ha", [("fp64", 1e-8), ("bf16x3", 1e-3 / EV)])
def test_evgw0_matches_oracle(gwc, prec, tol_ha):
    s = _all_state_system()
    ref, it_ref = G.evgw0(s, tol=1e-9)
    c = _ctx(gwc, s, prec)
    e, it = c.evgw0(tol=1e-9, max_iter=100)
    c.sync()
    e = e.cpu().numpy()
    assert np.max(np.abs(e - ref)) < tol_ha, (np.max(np.abs(e - ref)), it, it_ref)
    assert abs(it - it_ref) <= 2
    c.close()


def test_g_energies_in_sigma_core_match_oracle(gwc):
    s = _all_state_system()
    rng = np.random.default_rng(3)
    eps_t = s.eps + rng.uniform(-0.05, 0.05, s.n_states)
    st = s.with_g_energies(eps_t)
    w = np.array([-0.95, -0.5, 0.05, 0.8, 1.7])
    c = _ctx(gwc, s, "fp64")
    c.set_g_energies(eps_t)
    sig, _, _ = c.sigma_core(w)
    c.sync()
    got = sig[..., 0].cpu().numpy() + 1j * sig[..., 1].cpu().numpy()
    ref = np.stack([st.sigma_c(float(x))[0] for x in w], axis=1)
    assert np.max(np.abs(got - ref)) < 1e-8
    c.set_g_energies(None)  # back to the input energies in G
    sig0, _, _ = c.sigma_core(w)
    c.sync()
    got0 = sig0[..., 0].cpu().numpy() + 1j * sig0[..., 1].cpu().numpy()
    ref0 = np.stack([s.sigma_c(float(x))[0] for x in w], axis=1)
    assert np.max(np.abs(got0 - ref0)) < 1e-8
    c.close()


def test_virtual_cores_rejected_where_occupied_cores_are_needed(gwc):
    s = _all_state_system()
    c = _ctx(gwc, s, "fp64")
    with pytest.raises(gwc.GwcError) as err:
        c.qp_solve()
    assert err.value.status == 1
    c.close()


def test_evgw0_stop_without_convergence_matches_oracle(gwc):
    """Two steps cannot reach 1e-14 Ha: the oracle raises, the library reports GWC_ERR_NOT_CONVERGED, and
    the last iterate is the oracle's second iterate."""
    s = _all_state_system()
    with pytest.raises(G.NotConverged):
        G.evgw0(s, tol=1e-14, max_iter=2, on_fail="raise")
    ref, it_ref = G.evgw0(s, tol=1e-14, max_iter=2)
    assert it_ref == 2
    c = _ctx(gwc, s, "fp64")
    e = torch.empty(s.n_states, dtype=torch.float64, device="cuda")
    with pytest.raises(gwc.GwcError) as err:
        c.evgw0(tol=1e-14, max_iter=2, out=e)
    assert err.value.status == 5
    assert np.max(np.abs(e.cpu().numpy() - ref)) < 1e-8
    c.close()
