"""Writes tests/golden/pentacene_oracle.json: FP64 oracle values for the pentacene-sized workload.

Calls only the oracle (and the seeded input generator). The oracle is slow at this size (about 25 s
per residue build on 8 CPU cores), so it covers a bounded subset:
  * Hedin shifts dH_n = Re Sigma^c_n(eps_n) + Sigma^x_n - v^xc_n of cores 0, 11 and 21; with the
    default v^xc = Sigma^x the G_dH W0 QP energy is eps_n + dH_n (eq QPGWC), so dH gives the QP gate;
  * Sigma^c of all 22 cores at two grid frequencies (indices 100 and 700 of the 800-point grid);
  * with --dec: the DIAG-decoupled Im Sigma (Eq. cd_sigma_imaginary_decoupled) of cores 0, 11 and 21 at
    8 points of the relative grid nu_j = linspace(-25 eV, 5 eV, 800) (absolute w = eps_n + nu_j), the
    values the spectra of the request mode start from (one dielectric solve per core and point),
    added to an existing file under "dec_rel".
The file is rewritten after every result, so a partial run leaves the values it finished (the
lists "cores"/"dH" and "omega_idx"/"points" name what is present).
Run: python tests/golden/make_pentacene_golden.py [--dec]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import gwc_oracle as G  # noqa: E402
from paper_2412_17132_gb300 import synth  # noqa: E402

CORES = [0, 11, 21]
OMEGA_IDX = [100, 700]
DEC_NU_IDX = [20, 111, 203, 294, 386, 477, 569, 660]


def add_decoupled(out_path):
    import numpy as np

    t0 = time.time()
    with open(out_path) as f:
        res = json.load(f)
    mol = synth.pentacene()
    s = G.System.from_molecule(mol)
    nu = np.linspace(-25.0 / synth.HARTREE_EV, 5.0 / synth.HARTREE_EV, 800)
    own = list(range(mol.n_core))
    dec = res.get("dec_rel", {"nu_idx": DEC_NU_IDX, "cores": CORES, "values": []})
    for k, c in enumerate(CORES):
        if k < len(dec["values"]):
            continue
        row = [float(s.im_sigma_dec_group(float(mol.eps[c] + nu[j]), own, cores=[c])[c]) for j in DEC_NU_IDX]
        dec["values"].append(row)
        res["dec_rel"] = dec
        with open(out_path + ".tmp", "w") as f:
            json.dump(res, f, indent=1)
        os.replace(out_path + ".tmp", out_path)
        print(f"core {c}: decoupled Im Sigma at {len(DEC_NU_IDX)} points ({time.time() - t0:.0f} s)", flush=True)


def main(out_path):
    t0 = time.time()
    mol = synth.pentacene()
    s = G.System.from_molecule(mol)
    t_gen = time.time() - t0
    print(f"generated ({t_gen:.0f} s)", flush=True)
    s.w_imag_table()
    t_tab = time.time() - t0
    print(f"imaginary-axis table ({t_tab:.0f} s)", flush=True)
    sx = s.sigma_x()
    res = {"workload": "pentacene-sized synthetic molecule (synth.pentacene(), seed 0)", "cores": [],
           "omega_idx": [], "sigma_x": [float(v) for v in sx], "eps": [], "dH": [], "points": []}

    def save():
        # written after every result, so an interrupted run keeps what it finished
        res["seconds"] = {"generate": t_gen, "imag_table": t_tab - t_gen, "total": time.time() - t0}
        with open(out_path + ".tmp", "w") as f:
            json.dump(res, f, indent=1)
        os.replace(out_path + ".tmp", out_path)

    for c in CORES:
        sig = s.sigma_c_core(c, float(mol.eps[c]))
        res["cores"].append(c)
        res["eps"].append(float(mol.eps[c]))
        res["dH"].append(float(sig.real))  # + Sigma^x - v^xc = 0 with the default v^xc
        save()
        print(f"core {c}: dH = {res['dH'][-1]:.12f} Ha ({time.time() - t0:.0f} s)", flush=True)
    for j in OMEGA_IDX:
        sg, dec = s.sigma_c(float(mol.omega[j]))
        res["omega_idx"].append(j)
        res["points"].append({"omega": float(mol.omega[j]), "sigma_c": [[float(v.real), float(v.imag)] for v in sg],
                              "im_sigma_dec": [float(v) for v in dec]})
        save()
        print(f"omega[{j}] done ({time.time() - t0:.0f} s)", flush=True)

if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    path = args[0] if args else os.path.join(os.path.dirname(os.path.abspath(__file__)), "pentacene_oracle.json")
    if "--dec" in sys.argv:
        add_decoupled(path)
    else:
        main(path)
