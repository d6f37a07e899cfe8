"""Write geometric_L16.txt: the closed form of a geometric convolution, exactly.

For f_j = a^j and g_j = b^j (j < L) the first L outputs of the linear
convolution are h_k = sum_{j<=k} a^j b^(k-j) = (a^(k+1) - b^(k+1)) / (a - b).
The values are evaluated in exact rational arithmetic (fractions.Fraction) and
written with 20 significant digits; no code of the oracle or of the library is
used.  a = 0.9995, b = -0.999 (well separated, so the closed form is well
conditioned)."""
import os
from fractions import Fraction

A = Fraction(9995, 10000)
B = Fraction(-999, 1000)
L = 16


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "geometric_L16.txt")
    with open(out, "w") as fh:
        fh.write("# closed form h_k = (a^(k+1) - b^(k+1)) / (a - b), a = 0.9995, b = -0.999, k < 16\n")
        fh.write("# exact rational evaluation by tests/golden/make_geometric.py\n")
        for k in range(L):
            h = (A ** (k + 1) - B ** (k + 1)) / (A - B)
            fh.write(f"{k} {float(h):.20e} {h.numerator}/{h.denominator}\n")


if __name__ == "__main__":
    main()
