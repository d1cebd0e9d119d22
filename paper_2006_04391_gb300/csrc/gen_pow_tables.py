"""Writes pow_tables.inc: the constants of the table-driven FP64 power in
fpow.cuh, each the double nearest to its mathematical definition (evaluated
with Python's decimal module at 50 digits, then rounded once):

  kPowRcp[i]  = 1 / (1 + i/128)                       i = 0..127
  kPowLog2[i] = log2(1 + i/128)
  kPowExp2[i] = 2^(i/128)
  kPowLnC[k]  = (-1)^(k+1) / (k ln 2)                 k = 1..7   (log2(1+t) series)
  kPowExpC[k] = (ln 2)^k / k!                         k = 0..6   (2^r series)

Run from this directory: python gen_pow_tables.py
"""
import decimal
import os

D = decimal.Decimal
decimal.getcontext().prec = 50
LN2 = D(2).ln()


def h(x):
    return float(str(x)).hex()


def main():
    rcp = [D(1) / (D(1) + D(i) / 128) for i in range(128)]
    lg2 = [(D(1) + D(i) / 128).ln() / LN2 for i in range(128)]
    ex2 = [(LN2 * D(i) / 128).exp() for i in range(128)]
    lnc = [D((-1) ** (k + 1)) / (D(k) * LN2) for k in range(1, 8)]
    fact = 1
    exc = []
    for k in range(7):
        fact = fact * k if k > 0 else 1
        exc.append(LN2 ** k / D(fact))
    out = ["// Generated by gen_pow_tables.py; do not edit."]
    for name, vals in (("kPowRcp", rcp), ("kPowLog2", lg2), ("kPowExp2", ex2), ("kPowLnC", lnc), ("kPowExpC", exc)):
        out.append("GSM_POW_TABLE(%s, %d, {" % (name, len(vals)))
        for i in range(0, len(vals), 4):
            out.append("    " + ", ".join(h(v) for v in vals[i:i + 4]) + ",")
        out.append("})")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pow_tables.inc")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
