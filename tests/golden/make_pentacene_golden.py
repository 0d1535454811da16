"""Writes tests/golden/pentacene_oracle.json: FP64 oracle values for the pentacene-sized workload.

Calls only the oracle (and the seeded input generator). The oracle is slow at this size (about 25 s
per residue build on 8 CPU cores), so it covers a bounded subset:
  * Hedin shifts dH_n = Re Sigma^c_n(eps_n) + Sigma^x_n - v^xc_n of cores 0, 11 and 21; with the
    default v^xc = Sigma^x the G_dH W0 QP energy is eps_n + dH_n (eq QPGWC), so dH gives the QP gate;
  * Sigma^c of all 22 cores at two grid frequencies (indices 100 and 700 of the 800-point grid).
The file is rewritten after every result, so a partial run leaves the values it finished (the
lists "cores"/"dH" and "omega_idx"/"points" name what is present).
Run: python tests/golden/make_pentacene_golden.py
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
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "pentacene_oracle.json"))
