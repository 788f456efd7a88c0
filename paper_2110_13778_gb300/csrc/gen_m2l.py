"""Generate m2l_unrolled.cuh: straight-line MtL contraction bodies for fixed Taylor orders.

For a fixed order P the MtL sum of eqcoeff, written as
    a! lam^a = sum_{|a| + |b| <= P} D^{a+b} G(d) * M^b,   M^b = (-1)^|b| m^b / b!,
has a fixed set of (gamma = a + b, a, b) triples. Emitting them as explicit statements lets
the compiler keep the local coefficients in registers. Each body handles the multi-indices
a in one range [a0, a1) (the coefficients can be split into passes of at most SPLIT so
that one pass fits in registers), walks gamma in layout order, loads D^gamma from the
interleaved slot layout (Dl[gamma * 32]) in groups of GROUP so that several loads are in
flight before their values are used, and reads the scaled moments from shared memory
(Ms[b * 32], the interleaved chunk layout).

Run: python gen_m2l.py > m2l_unrolled.cuh  (the output is committed beside this script).
"""

ORDERS = (4, 6, 8)
SPLIT = 165
GROUP = 4


def multi_indices(p):
    out = []
    for n in range(p + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                out.append((a, b, n - a - b))
    return out


def passes(T):
    return [(a0, min(T, a0 + SPLIT)) for a0 in range(0, T, SPLIT)]


def body(P, a0, a1):
    idx = multi_indices(P)
    pos = {t: i for i, t in enumerate(idx)}
    work = []  # (gamma, [(alpha - a0, beta)])
    for g, gm in enumerate(idx):
        splits = []
        for ia in range(a0, a1):
            al = idx[ia]
            be = (gm[0] - al[0], gm[1] - al[1], gm[2] - al[2])
            if min(be) >= 0:
                splits.append((ia - a0, pos[be]))
        if splits:
            work.append((g, splits))
    out = []
    for s in range(0, len(work), GROUP):
        grp = work[s:s + GROUP]
        for k, (g, _) in enumerate(grp):
            out.append(f"        d{k} = Dl[{g * 32}];")
        for k, (_, splits) in enumerate(grp):
            for ia, ib in splits:
                out.append(f"        L[{ia}] += d{k} * Ms[{ib * 32}];")
    return out


def main():
    lines = [
        "// Generated by gen_m2l.py -- straight-line MtL contraction bodies. Do not edit.",
        "#pragma once",
        "",
        f"#define M2L_SPLIT {SPLIT}",
        "",
        "template <int P, int PASS>",
        "struct M2LBody;",
        "",
        "template <int P>",
        "struct M2LPassCount;",
        "",
    ]
    for P in ORDERS:
        T = len(multi_indices(P))
        ps = passes(T)
        lines.append(f"template <>\nstruct M2LPassCount<{P}> {{\n    static constexpr int n = {len(ps)};\n}};\n")
        for k, (a0, a1) in enumerate(ps):
            lines += [
                "template <>",
                f"struct M2LBody<{P}, {k}> {{",
                "    template <class R>",
                "    static __device__ __forceinline__ void run(const R* __restrict__ Dl, const R* __restrict__ Ms, R* L)",
                "    {",
                "        R " + ", ".join(f"d{i}" for i in range(GROUP)) + ";",
            ]
            lines += body(P, a0, a1)
            lines += ["    }", "};", ""]
    print("\n".join(lines))


if __name__ == "__main__":
    main()
