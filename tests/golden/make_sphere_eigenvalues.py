"""Writes sphere_cfie_eigenvalues.txt: eigenvalues of the combined-field
operator 1/2 I + D - i eta S (Sec. 3, Eqs. extdir and comb_ref) on the unit
sphere for spherical harmonics of degree 0 and 1.

On the unit sphere every spherical harmonic of degree n is an eigenfunction
(addition theorem for exp(ik|x - y|)/(4 pi |x - y|)):
    S Y_n = i k j_n(k) h_n(k) Y_n,   (1/2 I + D) Y_n = i k^2 j_n'(k) h_n(k) Y_n,
so lambda_n = i k^2 j_n'(k) h_n(k) + eta k j_n(k) h_n(k), h_n = h_n^(1).
Here j_0, j_1 and h_0, h_1 are written out in elementary functions (no
special-function library), so the values are an independent route to the
closed form the oracle's convergence test uses.
"""
import cmath
import math
import os


def lam(n: int, k: float, eta: float) -> complex:
    s, c = math.sin(k), math.cos(k)
    e = cmath.exp(1j * k)
    if n == 0:
        j = s / k
        jp = (k * c - s) / (k * k)
        h = -1j * e / k
    elif n == 1:
        j = s / (k * k) - c / k
        jp = (2.0 * k * c + (k * k - 2.0) * s) / k ** 3
        h = -e / k * (1.0 + 1j / k)
    else:
        raise ValueError(n)
    return 1j * k * k * jp * h + eta * k * j * h


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sphere_cfie_eigenvalues.txt")
    with open(out, "w") as f:
        f.write("# eigenvalues of 1/2 I + D - i eta S on the unit sphere (Sec. 3); "
                "written by make_sphere_eigenvalues.py\n")
        f.write("# n k eta re im\n")
        for k, eta in ((1.0, 1.0), (2.0, 2.0)):
            for n in (0, 1):
                v = lam(n, k, eta)
                f.write(f"{n} {k:.1f} {eta:.1f} {v.real:.15e} {v.imag:.15e}\n")
