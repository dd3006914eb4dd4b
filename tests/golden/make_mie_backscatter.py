"""Writes mie_backscatter.txt: the Mie-series monostatic RCS of the spheres the
benchmark solves (the Sec. V-A check), from oracle/mie.py only.  Besides the
two workload spheres it draws (seed 5) the operator catalogue of the
benchmark's serving trace: spheres meshed at level 2 or 3 with
f log-uniform in [0.1, 100] GHz, k0 r uniform in [0.2, 1], sigma
log-uniform in [1e-2, 5.8e7] S/m and eps_r uniform in [1, 12] (the serving
configuration's material and frequency ranges on electrically small spheres).

    python tests/golden/make_mie_backscatter.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mie  # noqa: E402

# name, radius (m), frequency (Hz), eps_r, sigma (S/m)
SPHERES = [
    ("dielectric-sphere-1920", 1e-2, 3e9, 4.0, 0.0),
    ("lossy-sphere-30720", 1e-3, 10e9, 1.0, 5.8e7),
]


def serve_catalogue(k=6, seed=5):
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        f = 10 ** rng.uniform(8, 11)
        kr = rng.uniform(0.2, 1.0)
        a = kr * 299792458.0 / (2 * np.pi * f)
        sigma = 10 ** rng.uniform(-2, np.log10(5.8e7))
        er = rng.uniform(1, 12)
        out.append((f"serve-{i}-L{2 + i % 2}", float(a), float(f), float(er), float(sigma)))
    return out


def rows():
    for name, a, f, er, s in SPHERES + serve_catalogue():
        yield name, a, f, er, s, mie.backscatter_rcs(a, f, er, s)


def main():
    with open(os.path.join(HERE, "mie_backscatter.txt"), "w") as fh:
        fh.write("# Mie-series backscatter RCS (m^2), written by make_mie_backscatter.py (oracle/mie.py)\n")
        fh.write("# name radius_m freq_hz eps_r sigma_S_per_m rcs_m2\n")
        for r in rows():
            fh.write("%s %.17e %.17e %.17e %.17e %.17e\n" % r)


if __name__ == "__main__":
    main()
