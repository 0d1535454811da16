"""The seeded input generators: determinism, symmetry, recipe, and host/device equivalence."""
import numpy as np
import pytest

from paper_2412_17132_gb300 import synth


def test_deterministic_and_symmetric_core_block():
    a = synth.small(n_states=20, n_occ=5, n_core=2, n_aux=12, seed=4)
    b = synth.small(n_states=20, n_occ=5, n_core=2, n_aux=12, seed=4)
    assert np.array_equal(a.o_ov, b.o_ov) and np.array_equal(a.o_core, b.o_core)
    # O^P_{c c'} = O^P_{c' c} for two cores
    assert np.array_equal(a.o_core[0, 1], a.o_core[1, 0])


def test_energy_recipe_tiny():
    m = synth.tiny()
    assert m.eps[0] == -10.40 and np.all(np.diff(m.eps) >= 0)
    assert np.sum((m.eps >= -1.0) & (m.eps <= -0.25)) == 7
    assert np.sum(m.eps > 3.0) == 5
    assert m.omega.size == 400 and abs((m.omega[-1] - m.omega[0]) * synth.HARTREE_EV - 30.0) < 1e-9


def test_device_generator_equals_host_generator_on_cpu():
    torch = pytest.importorskip("torch")
    for kw in (dict(n_states=30, n_occ=5, n_core=2, n_aux=40, seed=5), dict(n_states=26, n_occ=4, n_core=1, n_aux=2100, seed=6)):
        h = synth.molecule("x", kw["n_states"], kw["n_occ"], kw["n_core"], kw["n_aux"], seed=kw["seed"], n_omega=10)
        d = synth.molecule_device("x", kw["n_states"], kw["n_occ"], kw["n_core"], kw["n_aux"], seed=kw["seed"], n_omega=10,
                                  device="cpu", exact_scale=True)
        assert np.array_equal(h.eps, d.eps)
        assert np.max(np.abs(d.o_ov.numpy() - h.o_ov)) <= 1e-13 * np.max(np.abs(h.o_ov))
        assert np.max(np.abs(d.o_core.numpy() - h.o_core)) <= 1e-13 * np.max(np.abs(h.o_core))
