"""Writes dtensor_R122.txt: the field tensors D, D_i, D_ij, D_ijk, D_ijkl of -1/R at
R = (1, 2, 2) (|R| = 3) as exact rationals, evaluated from the closed forms printed in
Sec. 2.1 of arXiv:2107.07166 (eqs. D, Di, Dij, Dijk, Dijkl).  Calls nothing but the
standard library."""
from fractions import Fraction as F
from itertools import product
import os

R = (F(1), F(2), F(2))
R2 = sum(c * c for c in R)          # 9
r = F(3)                            # sqrt(9)


def dl(i, j):
    return F(1) if i == j else F(0)


def D0():
    return -1 / r


def D1(i):
    return R[i] / r ** 3


def D2(i, j):
    return (-3 * R[i] * R[j] + dl(i, j) * R2) / r ** 5


def D3(i, j, k):
    return (15 * R[i] * R[j] * R[k] - 3 * R2 * (dl(i, j) * R[k] + dl(j, k) * R[i] + dl(i, k) * R[j])) / r ** 7


def D4(i, j, k, l):
    t = -105 * R[i] * R[j] * R[k] * R[l]
    t += 15 * R2 * (dl(i, j) * R[k] * R[l] + dl(i, l) * R[j] * R[k] + dl(i, k) * R[j] * R[l]
                    + dl(j, l) * R[i] * R[k] + dl(j, k) * R[i] * R[l] + dl(l, k) * R[i] * R[j])
    t += -3 * R2 * R2 * (dl(i, j) * dl(k, l) + dl(i, k) * dl(j, l) + dl(i, l) * dl(j, k))
    return t / r ** 9


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dtensor_R122.txt")
    with open(out, "w") as f:
        f.write("# Field tensors of -1/R at R = (1,2,2), exact, from the closed forms of\n")
        f.write("# arXiv:2107.07166 Sec. 2.1, eqs. D, Di, Dij, Dijk, Dijkl.\n")
        f.write("# columns: tensor indices (0=x,1=y,2=z, '-' for the scalar)  numerator  denominator\n")
        v = D0()
        f.write(f"- {v.numerator} {v.denominator}\n")
        for n, fn in ((1, D1), (2, D2), (3, D3), (4, D4)):
            for idx in product(range(3), repeat=n):
                v = fn(*idx)
                f.write(f"{','.join(map(str, idx))} {v.numerator} {v.denominator}\n")


if __name__ == "__main__":
    main()
