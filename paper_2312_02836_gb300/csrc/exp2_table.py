"""Print the table of expf64.cuh: S_j = 2^(j/32), j = 0..31, as double-double
pairs (lead = 2^(j/32) rounded to the nearest double, trail = the remainder
rounded to the nearest double), from mpmath at 200 bits, in the hexadecimal
float form of the header's NB_EXP2_TABLE macro.

    python paper_2312_02836_gb300/csrc/exp2_table.py
"""
import mpmath


def table():
    """[(lead, trail)] for j = 0..31."""
    mpmath.mp.prec = 200
    out = []
    for j in range(32):
        s = mpmath.mpf(2) ** (mpmath.mpf(j) / 32)
        lead = float(s)
        trail = float(s - mpmath.mpf(lead))
        out.append((lead, trail))
    return out


def hexf(v: float) -> str:
    """C hexadecimal float literal (Python's float.hex, 0x0.0p+0 for zero)."""
    return "0x0.0p+0" if v == 0.0 else v.hex()


if __name__ == "__main__":
    pairs = [hexf(v) for lt in table() for v in lt]
    lines = [", ".join(pairs[i:i + 4]) for i in range(0, 64, 4)]
    print("#define NB_EXP2_TABLE" + " " * 53 + "\\")
    for i, line in enumerate(lines):
        print("  " + line + (", \\" if i + 1 < len(lines) else ""))
