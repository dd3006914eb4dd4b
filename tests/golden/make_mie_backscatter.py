"""Writes mie_backscatter.txt: the Mie-series monostatic RCS of the spheres the
benchmark solves (the Sec. V-A check), from oracle/mie.py only.

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


def rows():
    for name, a, f, er, s in SPHERES:
        yield name, a, f, er, s, mie.backscatter_rcs(a, f, er, s)


def main():
    with open(os.path.join(HERE, "mie_backscatter.txt"), "w") as fh:
        fh.write("# Mie-series backscatter RCS (m^2), written by make_mie_backscatter.py (oracle/mie.py)\n")
        fh.write("# name radius_m freq_hz eps_r sigma_S_per_m rcs_m2\n")
        for r in rows():
            fh.write("%s %.6e %.6e %.6e %.6e %.17e\n" % r)


if __name__ == "__main__":
    main()
