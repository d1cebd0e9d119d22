"""Writes pow_tables.inc: the constants of the table-driven FP64 power in
fpow.cuh, each the double nearest to its mathematical definition (evaluated
with Python's decimal module at 50 digits, then rounded once):

  kPowRcp[i]  = 1 / (1 + i/128)                       i = 0..127
  kPowLog2[i] = log2(1 + i/128)
  kPowExp2[i] = 2^(i/128)
  kPowLnC[k]  = (-1)^(k+1) / (k ln 2)                 k = 1..7   (log2(1+t) series)
  kPowExpC[k] = (ln 2)^k / k!                         k = 0..6   (2^r series)

and dpow_tables.inc, the tables of the double-float power in dpow.cuh, each
value split into the float nearest to it (hi) and the float nearest to the
remainder (lo), so hi + lo is within 2^-48 of the definition:

  kDpRcp[i]  = 1 / (1 + i/128)                        i = 0..128
  kDpLog2[i] = log2(1 + i/128)                        i = 0..128
  kDpExp2[i] = 2^(i/128)                              i = 0..127
  kDpConst   = 1/ln 2, ln 2 (hi, lo each)

Run from this directory: python gen_pow_tables.py
"""
import decimal
import os

D = decimal.Decimal
decimal.getcontext().prec = 50
LN2 = D(2).ln()


def h(x):
    return float(str(x)).hex()


def f32(x):
    """The float nearest to the decimal x (via the nearest double: a double
    rounding can move hi by one ulp, which only changes the split)."""
    import struct
    return struct.unpack("f", struct.pack("f", float(str(x))))[0]


def split(x):
    hi = f32(x)
    lo = f32(x - D(repr(hi)))
    return hi, lo


def hf(v):
    return float(v).hex() + "f"


def write_df_tables(path):
    rcp = [D(1) / (D(1) + D(i) / 128) for i in range(129)]
    lg2 = [(D(1) + D(i) / 128).ln() / LN2 for i in range(129)]
    ex2 = [(LN2 * D(i) / 128).exp() for i in range(128)]
    cst = [D(1) / LN2, LN2]
    out = ["// Generated by gen_pow_tables.py; do not edit.  Pairs (hi, lo)."]
    for name, vals in (("kDpRcp", rcp), ("kDpLog2", lg2), ("kDpExp2", ex2), ("kDpConst", cst)):
        out.append("GSM_DPOW_TABLE(%s, %d, {" % (name, 2 * len(vals)))
        for i in range(0, len(vals), 3):
            out.append("    " + ", ".join("%s, %s" % tuple(hf(v) for v in split(x)) for x in vals[i:i + 3]) + ",")
        out.append("})")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


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
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "pow_tables.inc"), "w") as f:
        f.write("\n".join(out) + "\n")
    write_df_tables(os.path.join(here, "dpow_tables.inc"))


if __name__ == "__main__":
    main()
