"""Writes tests/golden/pentacene_oracle.json: FP64 oracle values for the pentacene-sized workload.

Calls only the oracle (and the seeded input generator). The oracle is slow at this size (about 25 s
per residue build on 8 CPU cores), so it covers a bounded subset:
  * Hedin shifts dH_n = Re Sigma^c_n(eps_n) + Sigma^x_n - v^xc_n of cores 0, 11 and 21; with the
    default v^xc = Sigma^x the G_dH W0 QP energy is eps_n + dH_n (eq QPGWC), so dH gives the QP gate;
  * Sigma^c of all 22 cores at two grid frequencies (indices 100 and 700 of the 800-point grid).
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
    res = {"workload": "pentacene-sized synthetic molecule (synth.pentacene(), seed 0)", "cores": CORES,
           "omega_idx": OMEGA_IDX, "sigma_x": [float(v) for v in sx], "eps": [float(mol.eps[c]) for c in CORES]}
    dh = []
    for c in CORES:
        sig = s.sigma_c_core(c, float(mol.eps[c]))
        dh.append(float(sig.real))  # + Sigma^x - v^xc = 0 with the default v^xc
        print(f"core {c}: dH = {dh[-1]:.12f} Ha ({time.time() - t0:.0f} s)", flush=True)
    res["dH"] = dh
    sig_pts = []
    for j in OMEGA_IDX:
        sg, dec = s.sigma_c(float(mol.omega[j]))
        sig_pts.append({"omega": float(mol.omega[j]), "sigma_c": [[float(v.real), float(v.imag)] for v in sg],
                        "im_sigma_dec": [float(v) for v in dec]})
        print(f"omega[{j}] done ({time.time() - t0:.0f} s)", flush=True)
    res["points"] = sig_pts
    res["seconds"] = {"generate": t_gen, "imag_table": t_tab - t_gen, "total": time.time() - t0}
    with open(out_path, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "pentacene_oracle.json"))
