"""Per-kernel timing of the three dominant kernel groups through the C-ABI, at a chosen width.

The polarizability build (chi0_pair_kernel, or chi0_tc_kernel with GWC_CHI0_KERNEL=single), the
complex-symmetric factorisation (per 64-column panel: ldlt_panel_kernel, ldlt_planes_kernel and the
batched ldlt_update_kernel; GWC_FACTOR=tc the one-CTA ldlt_tc_kernel) and the W-table forward
substitution (wtable_gemm_kernel; GWC_WTABLE=simt the SIMT ldlt_solve_kernel) of one context, timed by
the library's own CUDA events (`profile=True`): `gwc_screen` on `--freqs` complex frequencies
z = w + i eta per call (one chi0 launch, one factorisation, one border solve), then one imaginary-axis
W table (the real chi0 builds, the factorisations and the 33-node solve). The default width is the pentacene-sized one (N_aux = 4500,
N_occ = 73) with fewer virtual states (N_states = 350: N_ov = 20 221), so that a launch holds a few GB
and profiles in seconds; `--n-states 1300` gives the full pentacene N_ov = 89 571.

    python -m paper_2412_17132_gb300.kernel_bench [--n-states 350] [--freqs 8] [--reps 3] [--prec bf16x3]

Prints one JSON line per repetition with the per-phase milliseconds and the algorithmic rates from the
library's own flop counts (chi0: N_aux (N_aux + 1) N_ov per part, two parts per complex frequency).
Inputs come from the seeded device generator (synth.molecule_device).
"""
import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-states", type=int, default=350)
    ap.add_argument("--n-occ", type=int, default=73)
    ap.add_argument("--n-core", type=int, default=22)
    ap.add_argument("--n-aux", type=int, default=4500)
    ap.add_argument("--freqs", type=int, default=8, help="complex frequencies per screen call")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--prec", default="bf16x3", choices=["bf16x3", "bf16x3f64", "bf16", "fp32", "fp64"])
    ap.add_argument("--no-table", action="store_true", help="skip the imaginary-axis W table")
    args = ap.parse_args(argv)

    import torch

    from paper_2412_17132_gb300 import gwc, synth

    mol = synth.molecule_device("kernel_bench", args.n_states, args.n_occ, args.n_core, args.n_aux, seed=0)
    eps_d = torch.as_tensor(mol.eps, device="cuda")
    nb = args.freqs
    ctx = gwc.Context(eps_d, mol.n_occ, mol.core_idx, mol.o_ov, mol.o_core, prec=args.prec, eta=mol.eta,
                      n_im=mol.n_im, batch=nb, profile=True)
    n_ov = mol.n_occ * (mol.n_states - mol.n_occ)
    z = torch.tensor([[0.4 + 0.01 * k, mol.eta] for k in range(nb)], dtype=torch.float64, device="cuda")
    rhs = mol.o_core[mol.n_occ // 2].unsqueeze(0).expand(nb, -1, -1).contiguous()
    base = {"n_aux": args.n_aux, "n_ov": n_ov, "freqs": nb, "prec": args.prec}
    for it in range(args.reps):
        ctx.reset_stats()
        ctx.screen(z, rhs)
        ctx.sync()
        st = ctx.stats()
        print(json.dumps(dict(base, rep=it, chi0_ms=st["chi0_ms"], chi0_tflops=st["chi0_flop"] / st["chi0_ms"] / 1e9,
                              factor_ms=st["factor_ms"], factor_tflops=st["factor_flop"] / st["factor_ms"] / 1e9,
                              solve_ms=st["solve_ms"])), flush=True)
    if not args.no_table:
        ef = 0.5 * (mol.eps[mol.n_occ - 1] + mol.eps[mol.n_occ])
        ctx.reset_stats()
        ctx.sigma_core(np.array([ef]), want_dec=False)
        ctx.sync()
        st = ctx.stats()
        print(json.dumps(dict(base, table=True, n_im=mol.n_im + 1, chi0_ms=st["chi0_ms"], factor_ms=st["factor_ms"],
                              solve_ms=st["solve_ms"], solve_launches=st["solve_launches"])), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
