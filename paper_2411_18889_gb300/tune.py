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


def survey_vjp(lib, vjp_sizes, rules, log):
    """The VJP shapes, timed in their hot path: the adjoint sweep of a
    recorded leapfrog (nbody_leapfrog_vjp_tape: one VJP per force evaluation,
    most with the force at the same positions), equal masses as in the
    adjoint workload, 8 steps with checkpoints every 4.  The sweep takes its
    VJP shape from the table, so each shape is timed under a one-rule table
    (the force rules kept)."""
    import tempfile

    import torch

    import nbody_inputs as ni
    from . import api

    nv = 4
    K, ck = 8, 4
    force_rules = [l for l in rules if l.split()[0] == "force"]
    tmp = tempfile.mkdtemp()
    winners = []
    try:
        for n in vjp_sizes:
            p, v, m = ni.plummer(n, 4)
            M = torch.from_numpy(m.astype(np.float32)).cuda()
            P = torch.from_numpy(p).cuda()
            V = torch.from_numpy(v).cuda()
            tape = torch.empty(api.nbody_tape_bytes(n, K, ck), dtype=torch.uint8, device="cuda")
            api.nbody_leapfrog_record(P, V, M, 2.0 ** -7, 2.0 ** -8, K, ck, tape)
            gxT = torch.from_numpy(ni.gaussian((n, 3), 5)).cuda()
            zero = torch.zeros_like(gxT)
            gx0, gv0 = torch.empty_like(gxT), torch.empty_like(gxT)
            gm = torch.empty((n,), dtype=torch.float64, device="cuda")
            reps = 2 if n >= (1 << 18) else 3
            t = []
            for k in range(nv):
                path = os.path.join(tmp, f"vjp{k}.txt")
                with open(path, "w") as f:
                    f.write("\n".join(force_rules + [f"vjp 0 {k}"]) + "\n")
                if lib.nbody_tune_load(path.encode()) <= 0:
                    raise RuntimeError(f"the library rejected {path}")
                t.append(_time(lambda: api.nbody_leapfrog_vjp_tape(M, 2.0 ** -7, 2.0 ** -8, K, ck, tape, gxT, zero,
                                                                   gx0, gv0, gm), reps))
            k = int(np.argmin(t))
            winners.append(k)
            log(f"vjp sweep n={n}: " + " ".join(f"{i}:{(K + 1) * n * n / x / 1e9:.0f}" for i, x in enumerate(t))
                + f" Gint/s -> {k}")
    finally:
        import shutil
        shutil.rmtree(tmp, ignore_errors=True)
    return [f"vjp {n_min} {k}" for n_min, k in _rules(vjp_sizes, winners)]


def survey(sizes=(1024, 4096, 8192, 16384, 32768, 65536, 262144, 1048576),
           vjp_sizes=(1024, 4096, 8192, 16384, 32768, 65536, 262144),
           out=DEFAULT_OUT, log=print, kinds=("force", "vjp", "batched")):
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
    keep = []  # the current table's rules, for the kinds not surveyed
    if os.path.exists(out):
        keep = [l.strip() for l in open(out) if l.strip() and not l.startswith("#")]
    if "force" not in kinds:
        lines += [l for l in keep if l.split()[0] == "force"]
    for pot in ((0, 1) if "force" in kinds else ()):
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
    if "vjp" in kinds:
        lines += survey_vjp(lib, vjp_sizes, [l for l in lines if not l.startswith("#")], log)
    else:
        lines += [l for l in keep if l.split()[0] == "vjp"]
    # Batched: ragged families keyed by their largest system, each advanced a
    # few leapfrog steps in one persistent launch (the way ensembles run).
    nb_shapes = lib.nbody_num_batched_configs()
    fam_max, bwin = [], []
    if "batched" not in kinds:
        lines += [l for l in keep if l.split()[0] == "batched"]
    for nmax, nsys in (((128, 4096), (512, 2048), (1024, 1024), (4096, 512)) if "batched" in kinds else ()):
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
    for n_min, k in (_rules(fam_max, bwin) if "batched" in kinds else ()):
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
    ap.add_argument("--only", action="append", choices=["force", "vjp", "batched"],
                    help="survey only these kernels (repeatable); the others keep the rules of the table at --out")
    args = ap.parse_args(argv)
    print(survey(out=args.out, kinds=tuple(args.only) if args.only else ("force", "vjp", "batched")))
    return 0


if __name__ == "__main__":
    sys.exit(main())
