"""Writes alpha_lazy_cases.txt: population vectors (81 values, the oracle's direction order) at
which the entropic alpha of Eq. (delH) has alpha_max = min over x_i < 0 of -1 / x_i >= 5/2,
x = feq / f - 1.  In that regime the kernel evaluates Delta H(alpha_max) only once a root estimate
reaches alpha_max.  The first cases have no root before alpha_max (alpha = alpha_max); the others
have a root below it.  They are found by a seeded random search that calls only the oracle:
near-equilibrium populations with a few directions depleted (large positive x, a skewed
distribution whose root lies above 2) and a few raised (the negative x that set alpha_max).

    python tests/golden/make_alpha_lazy_cases.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rd3q81 as O  # noqa: E402

N_EACH = 2


def main():
    lat = O.velocity_set()
    rng = np.random.default_rng(13)
    found = {"alpha_max": [], "root": []}
    for _ in range(40000):
        d = rng.normal(0, 0.02, lat.q)
        k = rng.integers(1, 20)
        d[rng.choice(lat.q, k, replace=False)] = -rng.uniform(0.9, 0.999, k)
        j = rng.integers(1, 6)
        d[rng.choice(lat.q, j, replace=False)] = rng.uniform(0.5, 1.0, j)
        f = (lat.w * (1 + d))[:, None]
        rho, u, th = O.moments(f, lat)
        feq = O.entropic_equilibrium(rho, u, th, lat)[0]
        if not np.all(np.isfinite(feq)):
            continue
        x = (feq / f - 1)[:, 0]
        if x.min() >= 0 or -1 / x.min() < 2.5:
            continue
        amax = -1 / x.min()
        al = O.entropic_alpha(f, feq)[0]
        key = "alpha_max" if np.isclose(al, amax, rtol=1e-12) else "root"
        if len(found[key]) < N_EACH:
            found[key].append((amax, al, f[:, 0]))
        if all(len(v) >= N_EACH for v in found.values()):
            break
    path = os.path.join(HERE, "alpha_lazy_cases.txt")
    with open(path, "w") as fh:
        fh.write("# Entropic alpha (Eq. (delH)) with alpha_max >= 5/2: written by make_alpha_lazy_cases.py "
                 "(oracle only).\n# One case per line: 81 populations in the oracle's direction order.\n")
        for key in ("alpha_max", "root"):
            for amax, al, f in found[key]:
                fh.write(f"# {key}: alpha_max {amax:.12g}, oracle alpha {al:.12g}\n")
                fh.write(" ".join(repr(float(v)) for v in f) + "\n")
    print(path, {k: len(v) for k, v in found.items()})


if __name__ == "__main__":
    main()
