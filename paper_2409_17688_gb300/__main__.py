"""Command line for the library (each command one call of the C ABI).

  python -m paper_2409_17688_gb300 gamma2 --n 9 --m 1000          gamma_2(P_n x C_m)
  python -m paper_2409_17688_gb300 table --n 9 --kmax 200          gamma_2 for m = 3..kmax
  python -m paper_2409_17688_gb300 recurrence --n 12 [--ring 4]    (n0, a, b) of Table 4
  python -m paper_2409_17688_gb300 circuit --n 10                  the step's reuse circuit
  python -m paper_2409_17688_gb300 product --N 8192 --dtype u8 --seed 1 --inf-frac 0.4
  python -m paper_2409_17688_gb300 save --n 8 --kmax 12 --out powers.mpp   checkpoint A^1..A^kmax
  python -m paper_2409_17688_gb300 autotune [--out tiles.json]     tile table of this GPU

Every command prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import sys
import time


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2409_17688_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("gamma2")
    g.add_argument("--n", type=int, required=True)
    g.add_argument("--m", type=int, required=True)
    g.add_argument("--squaring", action="store_true", help="repeated squaring only")
    t = sub.add_parser("table")
    t.add_argument("--n", type=int, required=True)
    t.add_argument("--kmax", type=int, required=True)
    r = sub.add_parser("recurrence")
    r.add_argument("--n", type=int, required=True)
    r.add_argument("--klimit", type=int, default=64)
    r.add_argument("--ring", type=int, default=4)
    c = sub.add_parser("circuit")
    c.add_argument("--n", type=int, required=True)
    p = sub.add_parser("product")
    p.add_argument("--N", type=int, default=8192)
    p.add_argument("--dtype", choices=["i16", "u8"], default="i16")
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--inf-frac", type=float, default=0.4)
    s = sub.add_parser("save")
    s.add_argument("--n", type=int, required=True)
    s.add_argument("--kmax", type=int, required=True)
    s.add_argument("--out", required=True)
    a = sub.add_parser("autotune")
    a.add_argument("--out")
    args = ap.parse_args(argv)

    import paper_2409_17688_gb300 as mp
    t0 = time.perf_counter()
    if args.cmd == "gamma2":
        f = mp.mp_gamma2_squaring if args.squaring else mp.mp_gamma2_cylinder
        out = {"n": args.n, "m": args.m, "gamma2": f(args.n, args.m)}
    elif args.cmd == "table":
        tab = mp.mp_gamma2_table(args.n, args.kmax)
        out = {"n": args.n, "gamma2": {int(m): int(tab[m]) for m in range(3, args.kmax + 1)}}
    elif args.cmd == "recurrence":
        n0, a_, b, k = mp.mp_transfer_recurrence_stream(args.n, args.klimit, args.ring)
        out = {"n": args.n, "n0": n0, "a": a_, "b": b, "found_at_k": k}
    elif args.cmd == "circuit":
        out = dict(mp.mp_transfer_circuit_info(args.n), n=args.n)
    elif args.cmd == "product":
        import numpy as np
        import torch
        from paper_2409_17688_gb300 import synth
        dt = np.int16 if args.dtype == "i16" else np.uint8
        X = torch.from_numpy(synth.block_inf_matrix(args.N, args.N, args.seed, dt, inf_frac=args.inf_frac)).cuda()
        Y = torch.from_numpy(synth.block_inf_matrix(args.N, args.N, args.seed + 1, dt,
                                                    inf_frac=args.inf_frac)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Z = mp.mp_minplus_mul(X, Y)
        torch.cuda.synchronize()
        out = {"N": args.N, "dtype": args.dtype, "ms": round((time.perf_counter() - t0) * 1e3, 3),
               "z_min": int(Z.min().item()), "z_max": int(Z.max().item())}
    elif args.cmd == "save":
        P, _ = mp.mp_transfer_power_sequence(args.n, args.kmax)
        mp.mp_powers_save(args.out, args.n, 1, P)
        out = dict(mp.mp_powers_info(args.out), path=args.out)
    else:
        table = mp.mp_autotune()
        out = {"tile_table": table.tolist()}
        if args.out:
            with open(args.out, "w") as fh:
                json.dump(out, fh)
    out["seconds"] = round(time.perf_counter() - t0, 4)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
