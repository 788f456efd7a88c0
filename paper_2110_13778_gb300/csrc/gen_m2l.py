"""Generate m2l_unrolled.cuh: straight-line MtL contraction bodies for fixed Taylor orders.

For a fixed order P the MtL sum of eqcoeff, written as
    a! lam^a = sum_{|a| + |b| <= P} D^{a+b} G(d) * M^b,   M^b = (-1)^|b| m^b / b!,
has a fixed set of (gamma = a + b, a, b) triples. Emitting them as explicit statements lets
the compiler keep the local coefficients in registers. Each body handles the multi-indices
a in one range [a0, a1) (the order's coefficients are split into passes of at most 84 so
that one pass fits in registers), walks gamma in layout order, loads D^gamma once per pair
from the interleaved slot layout (Dl[gamma * 32]) and reads the scaled moments from shared
memory (Ms[b * 33]).

Run: python gen_m2l.py > m2l_unrolled.cuh  (the output is committed beside this script).
"""


def multi_indices(p):
    out = []
    for n in range(p + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                out.append((a, b, n - a - b))
    return out


ORDERS = (4, 6, 8)
SPLIT = 84


def passes(T):
    out = []
    a0 = 0
    while a0 < T:
        out.append((a0, min(T, a0 + SPLIT)))
        a0 += SPLIT
    return out


def main():
    lines = [
        "// Generated by gen_m2l.py -- straight-line MtL contraction bodies. Do not edit.",
        "#pragma once",
        "",
        "template <int P, int PASS>",
        "struct M2LBody;",
        "",
    ]
    for P in ORDERS:
        idx = multi_indices(P)
        pos = {t: i for i, t in enumerate(idx)}
        T = len(idx)
        ps = passes(T)
        lines.append(f"template <>\nstruct M2LPasses<{P}> {{ static constexpr int n = {len(ps)}; }};" if False else "")
        for k, (a0, a1) in enumerate(ps):
            lines.append("template <>")
            lines.append(f"struct M2LBody<{P}, {k}> {{")
            lines.append(f"    static constexpr int A0 = {a0}, A1 = {a1};")
            lines.append("    template <class R>")
            lines.append("    static __device__ __forceinline__ void run(const R* __restrict__ Dl, const R* __restrict__ Ms, R* L)")
            lines.append("    {")
            lines.append("        R d;")
            for g, gm in enumerate(idx):
                splits = []
                for ia in range(a0, a1):
                    al = idx[ia]
                    be = (gm[0] - al[0], gm[1] - al[1], gm[2] - al[2])
                    if min(be) < 0:
                        continue
                    splits.append((ia, pos[be]))
                if not splits:
                    continue
                lines.append(f"        d = Dl[{g * 32}];")
                for ia, ib in splits:
                    lines.append(f"        L[{ia - a0}] += d * Ms[{ib * 33}];")
            lines.append("    }")
            lines.append("};")
            lines.append("")
    lines.append("template <int P>")
    lines.append("struct M2LPassCount;")
    for P in ORDERS:
        T = len(multi_indices(P))
        lines.append(f"template <>\nstruct M2LPassCount<{P}> {{ static constexpr int n = {len(passes(T))}; }};")
    print("\n".join(l for l in lines if l is not None))


if __name__ == "__main__":
    main()
