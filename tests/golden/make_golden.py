"""Write the stored expected values under tests/golden/ (calls only oracle/).

disc_F10_hankel.json: u^ap of the unit disc at lambda z = 0.1 (Fresnel number
10, Sec. 2 eq. fn) at several radii rho, from the Hankel-type 1D reduction of
eq. fres (oracle.closed_forms.disc_off_axis) and, at rho = 0, from Appendix
eq. dauger with R(theta) = 1 (oracle.closed_forms.disc_on_axis).

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import closed_forms  # noqa: E402


def main():
    R, lz = 1.0, 0.1
    rho = [0.0, 0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 2.0, 2.1213203435596424]
    u = closed_forms.disc_off_axis(R, lz, rho, n_quad=6000)
    u0 = closed_forms.disc_on_axis(R, lz)
    out = {
        "citation": "arXiv:2010.05978 eq. fres (Sec. 2) reduced for a disc; "
                    "rho = 0 also from Appendix eq. dauger with R(theta) = R",
        "R": R, "lambda_z": lz,
        "rho": rho,
        "u_re": [float(v.real) for v in u],
        "u_im": [float(v.imag) for v in u],
        "u_axis_dauger": [float(u0.real), float(u0.imag)],
    }
    with open(os.path.join(HERE, "disc_F10_hankel.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
