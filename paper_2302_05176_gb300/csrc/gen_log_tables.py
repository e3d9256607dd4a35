"""Generate gm_log_tables.h: constants of the integer natural logarithm in gm_arith.cuh.

Method: table-driven logarithm (P. T. P. Tang, "Table-driven implementation of
the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990),
carried out in 64/128-bit integer fixed point instead of floating point:

    f in [1, 2),  j = top 8 fraction bits of f,  F_j = 1 + (j + 1/2)/256
    INV_j = RN(2^64 / F_j)                       (u64; 1/F_j to 64 bits)
    1 + r = f * INV_j / 2^64                      (exact 128-bit product, |r| < 2^-9)
    ln f  = ln(1 + r) - ln(INV_j / 2^64)          (an identity: no error from INV_j)

LNF_j = -ln(INV_j / 2^64) is tabulated to 2^-120 from the exact INV_j, so the only
rounding errors are those of the short series for ln(1 + r).  Every constant is
computed here from its mathematical definition with mpmath at 200 bits.

Run: python gen_log_tables.py > gm_log_tables.h
"""
import mpmath

mpmath.mp.prec = 200
TAB_BITS = 8
N = 1 << TAB_BITS


def rn(x):
    return int(mpmath.nint(x))


def main():
    out = []
    out.append("// gm_log_tables.h -- generated by gen_log_tables.py; do not edit.")
    out.append("// Constants of the integer logarithm (Tang's table-driven method in fixed point).")
    out.append("#pragma once")
    out.append("#include <cstdint>")
    out.append("namespace gm {")
    out.append("constexpr int LOG_TAB_BITS = %d;" % TAB_BITS)
    inv, lnf_hi, lnf_lo = [], [], []
    for j in range(N):
        F = 1 + (mpmath.mpf(j) + mpmath.mpf(1) / 2) / N
        I = rn(mpmath.mpf(2) ** 64 / F)
        assert 2 ** 63 < I < 2 ** 64
        L = -mpmath.log(mpmath.mpf(I) / mpmath.mpf(2) ** 64)
        Li = rn(L * mpmath.mpf(2) ** 120)
        assert 0 <= Li < 2 ** 128
        inv.append(I)
        lnf_hi.append(Li >> 64)
        lnf_lo.append(Li & (2 ** 64 - 1))
    ln2 = rn(mpmath.log(2) * mpmath.mpf(2) ** 120)

    def arr(name, vals):
        # indexed per lane: global memory, read through the read-only cache
        out.append("__device__ const uint64_t %s[%d] = {" % (name, len(vals)))
        for i in range(0, len(vals), 4):
            out.append("    " + ", ".join("0x%016xull" % v for v in vals[i:i + 4]) + ",")
        out.append("};")

    arr("LOG_INV", inv)
    arr("LOG_LNF_HI", lnf_hi)
    arr("LOG_LNF_LO", lnf_lo)
    out.append("constexpr uint64_t LN2_120_HI = 0x%016xull;  // ln 2 * 2^120, rounded" % (ln2 >> 64))
    out.append("constexpr uint64_t LN2_120_LO = 0x%016xull;" % (ln2 & (2 ** 64 - 1)))
    # ln(1+r) = r - r^2/2 + r^3 B(r),  B = 1/3 - r/4 + r^2 (1/5 - r/6 + r^2/7)
    out.append("// (lane-uniform constants) ln(1+r) = r - r^2/2 + r^3 (1/3 - r/4 + r^2 (1/5 - r/6 + r^2/7))")
    out.append("constexpr int64_t LOG_C3 = %dll;  // 2^62 / 3" % rn(mpmath.mpf(2) ** 62 / 3))
    out.append("constexpr int32_t LOG_C5 = %d;  // 2^31 / 5" % rn(mpmath.mpf(2) ** 31 / 5))
    out.append("constexpr int32_t LOG_C6 = %d;  // 2^31 / 6" % rn(mpmath.mpf(2) ** 31 / 6))
    out.append("constexpr int32_t LOG_C7 = %d;  // 2^31 / 7" % rn(mpmath.mpf(2) ** 31 / 7))
    # -ln(1-w) = w P(w), P(w) = sum_{i>=0} w^i/(i+1) ; coefficients at scale 2^63
    p = [rn(mpmath.mpf(2) ** 63 / (i + 1)) for i in range(9)]
    out.append("// 2^63 / (i+1) for i = 0..8: P(w) = 1 + w/2 + ... + w^8/9 of -ln(1-w) = w P(w)")
    out.append("__device__ __constant__ uint64_t LOG1M_P[9] = {" + ", ".join("0x%016xull" % v for v in p) + "};")
    out.append("}  // namespace gm")
    print("\n".join(out))


if __name__ == "__main__":
    main()
