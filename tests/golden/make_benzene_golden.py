"""Writes tests/golden/benzene_oracle.json: FP64 oracle values for the benzene-sized workload.

Calls only the oracle (and the seeded input generator). Contents:
  * the DIAG-decoupled Im Sigma of all 6 cores on the whole 800-point grid (Eq.
    cd_sigma_imaginary_decoupled: f_n Im W^c_nn(|eps_n - w| + i eta), one dielectric solve per core and
    frequency; the oracle's group form with every core in its own group is the DIAG form), the input of
    the cumulant spectra whose A(w) and satellite positions the GPU parity test gates;
  * Sigma^c (Eq. cd_terms: -I + R, all residue states) of all 6 cores at 16 grid frequencies spread over
    the window.
Run: python tests/golden/make_benzene_golden.py   (about 10 minutes on 8 CPU cores)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import gwc_oracle as G  # noqa: E402
from paper_2412_17132_gb300 import synth  # noqa: E402

SIGMA_IDX = [int(v) for v in np.linspace(0, 799, 16).round()]


def main(out_path):
    t0 = time.time()
    mol = synth.benzene()
    s = G.System.from_molecule(mol)
    own = list(range(mol.n_core))  # every core in its own group: the DIAG form
    dec = np.zeros((mol.n_core, mol.omega.size))
    for j, w in enumerate(mol.omega):
        dec[:, j] = s.im_sigma_dec_group(float(w), own)
        if j % 100 == 0:
            print(f"decoupled Im Sigma: {j}/{mol.omega.size} ({time.time() - t0:.0f} s)", flush=True)
    sig = []
    for j in SIGMA_IDX:
        sg, _ = s.sigma_c(float(mol.omega[j]))
        sig.append([[float(v.real), float(v.imag)] for v in sg])
    res = {"workload": "benzene-sized synthetic molecule (synth.benzene(), seed 0)",
           "omega": [float(v) for v in mol.omega],
           "eps_core": [float(mol.eps[c]) for c in mol.core_idx],
           "im_sigma_dec": dec.tolist(),
           "sigma_idx": SIGMA_IDX, "sigma_c": sig,
           "seconds": time.time() - t0}
    with open(out_path + ".tmp", "w") as f:
        json.dump(res, f)
    os.replace(out_path + ".tmp", out_path)
    print(f"done ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "benzene_oracle.json"))
