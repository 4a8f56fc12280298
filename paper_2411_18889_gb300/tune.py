"""Parameter survey of the kernel shapes on the current GPU.

Miki & Hanawa chose the threads per block of their N-body kernel by a
parameter survey on each machine (Sec. III.A).  This module does the same for
every compiled shape of the force, VJP and batched kernels: it times each shape
at a ladder of sizes through the C ABI -- the force without the potential in
a leapfrog of 4 steps (its hot path: evaluations and the packs between them),
with the potential in single nbody_accel calls -- and writes the winners as a
table the library reads
(``nbody_tune.txt`` beside libnbody.so, or the file named by NBODY_TUNE_FILE).

    python -m paper_2411_18889_gb300.tune --out paper_2411_18889_gb300/nbody_tune.txt
"""
from __future__ import annotations

import argparse
import datetime
import os
import sys

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(PKG, "nbody_tune.txt")


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / 1e3)
    return best


def _rules(sizes, winners):
    """Size ladder -> rules: each size owns n from the midpoint below it."""
    out = []
    for i, (n, k) in enumerate(zip(sizes, winners)):
        n_min = 0 if i == 0 else (sizes[i - 1] + n) // 2
        if out and out[-1][1] == k:
            continue
        out.append((n_min, k))
    return out


def survey(sizes=(1024, 4096, 16384, 32768, 65536, 262144, 1048576),
           vjp_sizes=(1024, 4096, 16384, 32768, 65536, 262144),
           out=DEFAULT_OUT, log=print):
    import torch

    import nbody_inputs as ni
    from . import api
    from ._lib import load

    lib = load()
    lines = [f"# kernel-shape table written by paper_2411_18889_gb300.tune on "
             f"{torch.cuda.get_device_name(0)}, {datetime.date.today().isoformat()}",
             "# kind pot n_min shape (force), kind n_min shape (vjp), kind n_min shape (batched; n_min compared "
             "with the largest system)"]
    nf = lib.nbody_num_configs()
    for pot in (0, 1):
        winners = []
        for n in sizes:
            p, v, m = ni.plummer(n, 3, masses="loguniform", offset=ni.plummer_offset())
            P = torch.from_numpy(p).cuda()
            M = torch.from_numpy(m.astype(np.float32)).cuda()
            reps = 2 if n >= (1 << 19) else 5
            if pot:
                # the potential is wanted by single evaluations (nbody_accel, nbody_energy)
                acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
                pt = torch.empty((n,), dtype=torch.float32, device="cuda")
                evals = 1
                t = [_time(lambda k=k: api.nbody_accel(P, M, 2.0 ** -9, acc, pt, config=k), reps)
                     for k in range(nf)]
            else:
                # without it the hot path is the leapfrog: 4 steps (5 evaluations and their packs)
                V0 = torch.from_numpy(v).cuda()
                X, V = P.clone(), V0.clone()
                evals = 5

                def run(k):
                    X.copy_(P)
                    V.copy_(V0)
                    api.nbody_leapfrog(X, V, M, 2.0 ** -9, 2.0 ** -9, 4, config=k)

                t = [_time(lambda k=k: run(k), reps) for k in range(nf)]
            k = int(np.argmin(t))
            winners.append(k)
            log(f"force pot={pot} n={n}: " + " ".join(f"{i}:{evals * n * n / x / 1e9:.0f}" for i, x in enumerate(t))
                + f" Gint/s -> {k}")
        for n_min, k in _rules(sizes, winners):
            lines.append(f"force {pot} {n_min} {k}")
    nv = 4
    winners = []
    for n in vjp_sizes:
        p, _, m = ni.plummer(n, 4, masses="loguniform")
        P = torch.from_numpy(p).cuda()
        M = torch.from_numpy(m.astype(np.float32)).cuda()
        lam = torch.from_numpy(ni.gaussian((n, 3), 5).astype(np.float32)).cuda()
        gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        gm = torch.empty((n,), dtype=torch.float32, device="cuda")
        t = [_time(lambda k=k: api.nbody_accel_vjp(P, M, 2.0 ** -7, lam, None, gp, gm, config=k), 3)
             for k in range(nv)]
        k = int(np.argmin(t))
        winners.append(k)
        log(f"vjp n={n}: " + " ".join(f"{i}:{n * n / x / 1e9:.0f}" for i, x in enumerate(t)) + f" Gint/s -> {k}")
    for n_min, k in _rules(vjp_sizes, winners):
        lines.append(f"vjp {n_min} {k}")
    # Batched: ragged families keyed by their largest system, each advanced a
    # few leapfrog steps in one persistent launch (the way ensembles run).
    nb_shapes = 4
    fam_max, bwin = [], []
    for nmax, nsys in ((128, 4096), (512, 2048), (1024, 1024), (4096, 512)):
        off, pos, vel, mass, eps = ni.ragged_batch(nsys=nsys, seed=4, nmin=max(16, nmax // 64), nmax=nmax)
        O = torch.from_numpy(off).cuda()
        P0 = torch.from_numpy(pos.astype(np.float32)).cuda()
        V0 = torch.from_numpy(vel.astype(np.float32)).cuda()
        M = torch.from_numpy(mass.astype(np.float32)).cuda()
        E = torch.from_numpy(eps.astype(np.float32)).cuda()
        P, V = P0.clone(), V0.clone()

        def run(k):
            P.copy_(P0)
            V.copy_(V0)
            api.nbody_leapfrog_batched(O, P, V, M, E, 2.0 ** -8, 8, config=k)

        t = [_time(lambda k=k: run(k), 3) for k in range(nb_shapes)]
        k = int(np.argmin(t))
        log(f"batched max {nmax}: " + " ".join(f"{i}:{x * 1e3:.2f}ms" for i, x in enumerate(t)) + f" -> {k}")
        fam_max.append(int(np.diff(off).max()))
        bwin.append(k)
    for n_min, k in _rules(fam_max, bwin):
        lines.append(f"batched {n_min} {k}")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    rc = lib.nbody_tune_load(out.encode())
    if rc <= 0:
        raise RuntimeError(f"the library rejected the table it was given ({rc})")
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)
    print(survey(out=args.out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
