"""Write adjoint_fd_n16384.json: FP64 central finite differences of the
adjoint workload's loss on 32 seeded coordinates, from the oracle alone.

The workload: N = 16384 Plummer sphere (seed 5), eps = 2^-7, dt = 2^-8,
K = 64 kick-drift-kick steps, loss L = sum_i m_i |x_i(T) - y_i|^2 with
y = x(0) + N(0, 0.05^2) offsets (seed 6).  For each of 32 coordinates drawn
from the 7N inputs (x0 components, v0 components, masses; seeded subsample,
seed 7) the derivative is (L(q + h) - L(q - h)) / 2h with h = 1e-6, each L one
FP64 oracle leapfrog run.  Nothing here touches the CUDA library: the values
are expectations for the GPU adjoint (tests/test_gpu_adjoint.py, bench.py).

Run from the repository root:  python tests/golden/make_adjoint_fd.py
(64 oracle runs of 65 force evaluations at N = 16384: about 1.1e12 FP64
interactions, minutes on a multicore host).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import nbody_inputs as ni  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "adjoint_fd_n16384.json")
H = 1e-6
NCOORD = 32
COORD_SEED = 7


def input_fingerprint(pos, vel, mass, target) -> dict:
    """Sums of |x| and a few entries of each input array.  numpy's transcendental
    functions (pow, exp, sin, cos) may differ in the last bit between x86 and
    Arm builds, so the generated inputs agree only to ~1e-16 relative across
    machines; a reader compares these numbers with a 1e-12 relative tolerance,
    which any real change of the inputs (another seed, another body) exceeds
    by orders of magnitude."""
    fp = {}
    for name, a in (("pos", pos), ("vel", vel), ("mass", mass), ("target", target)):
        a = np.asarray(a, dtype=np.float64).reshape(-1)
        fp[name] = {"sum_abs": float(np.abs(a).sum()), "head": [float(x) for x in a[:4]],
                    "tail": [float(x) for x in a[-4:]]}
    return fp


def main():
    w = ni.adjoint_case()
    n, K = w.n, w.steps
    p, v, m, y = w.pos, w.vel, w.mass, w.extra["target"]

    def loss(x0, v0, mass):
        xT, _, _ = oracle.leapfrog(x0, v0, mass, w.eps, w.dt, K)
        return float((mass[:, None] * (xT - y) ** 2).sum())

    pick = ni.subsample(7 * n, NCOORD, COORD_SEED)
    rows = []
    t0 = time.time()
    for q in pick:
        kind, body = divmod(int(q), n)  # 0..2: x0 component, 3..5: v0 component, 6: mass
        xp, vp, mp = p.copy(), v.copy(), m.copy()
        xm, vm, mm = p.copy(), v.copy(), m.copy()
        if kind < 3:
            xp[body, kind] += H
            xm[body, kind] -= H
        elif kind < 6:
            vp[body, kind - 3] += H
            vm[body, kind - 3] -= H
        else:
            mp[body] += H
            mm[body] -= H
        lp, lm = loss(xp, vp, mp), loss(xm, vm, mm)
        rows.append({"coord": int(q), "kind": ["x0", "v0", "m"][min(kind // 3, 2)], "body": body,
                     "component": kind % 3 if kind < 6 else 0, "L_plus": lp, "L_minus": lm,
                     "fd": (lp - lm) / (2 * H)})
        print(f"{len(rows)}/{NCOORD} {rows[-1]['kind']}[{body}] fd={rows[-1]['fd']:.12e} "
              f"({time.time() - t0:.0f} s)", flush=True)
    doc = {
        "what": "FP64 central finite differences of L = sum m |x(T) - y|^2 for the adjoint workload",
        "workload": {"n": n, "plummer_seed": 5, "target_seed": 6, "eps": w.eps, "dt": w.dt, "steps": K,
                     "masses": "equal, rounded to FP32", "target_sigma": 0.05},
        "h": H, "coord_seed": COORD_SEED,
        "coord_encoding": "q = kind * n + body; kind 0..2 x0[body][kind], 3..5 v0[body][kind-3], 6 m[body]",
        "inputs_fingerprint": input_fingerprint(p, v, m, y),
        "written_by": "tests/golden/make_adjoint_fd.py (oracle/ only)",
        "rows": rows,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
