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

M2LWarp<P, W> is the register-blocked two-warp variant used by the FP32 kernel: warp W
accumulates half of the local coefficients (equal FMA counts), the moments of a block of
MBLOCK multi-indices sit in registers, and each D^gamma is loaded once per block instead of
once per FMA, so the shared-memory loads per slot and kernel fall from 3168 to about 740
(both warps together) at P = 8, with about 170 registers per thread and no spills. Their
moments are read at Ms[b * 33] (rows padded to 33 words).

Run: python gen_m2l.py > m2l_unrolled.cuh  (the output is committed beside this script).
"""

from math import comb

ORDERS = (4, 6, 8)
SPLIT = 165
GROUP = 4
# two-warp register-blocked bodies (FP32 kernel): the local coefficients are split between two
# warps with equal FMA counts, and each warp holds the moments of MBLOCK multi-indices at a
# time in registers
NWARP = 2
MBLOCK = {4: 35, 6: 84, 8: 84}
# row stride of the moments in shared memory for the two-warp bodies: 33, so that the kernel
# can write one source's moments (lanes over b) without bank conflicts
MSTRIDE = 33


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


def warp_sets(P):
    """Split the multi-indices a between NWARP warps so that each gets the same number of
    (a, b) pairs: a pairs with C(P - |a| + 3, 3) moments, so low orders are heavy. Greedy,
    heaviest first, ties to the lower warp; each set in layout order."""
    idx = multi_indices(P)
    wt = [comb(P - sum(a) + 3, 3) for a in idx]
    load = [0] * NWARP
    sets = [[] for _ in range(NWARP)]
    for i in sorted(range(len(idx)), key=lambda i: (-wt[i], i)):
        k = load.index(min(load))
        load[k] += wt[i]
        sets[k].append(i)
    return [sorted(x) for x in sets]


def body_blocked(P, mb, aset):
    """Register-blocked form for the local coefficients a in `aset` (held as L[k], k the
    position in aset): the moments M^b of one block of mb multi-indices are loaded into
    registers once; then each D^gamma that pairs with the block is loaded once and every
    pair (a = gamma - b in aset, b in the block) is accumulated. Shared-memory loads per slot
    drop from one per FMA to (#gamma reached per block) + (#moments used)."""
    idx = multi_indices(P)
    pos = {t: i for i, t in enumerate(idx)}
    loc = {a: k for k, a in enumerate(aset)}
    T = len(idx)
    out = []
    for b0 in range(0, T, mb):
        blk = list(range(b0, min(T, b0 + mb)))
        work, used = [], set()
        for g, gm in enumerate(idx):
            prs = []
            for k, b in enumerate(blk):
                be = idx[b]
                al = (gm[0] - be[0], gm[1] - be[1], gm[2] - be[2])
                if min(al) >= 0 and pos[al] in loc:
                    prs.append((loc[pos[al]], k))
                    used.add(k)
            if prs:
                work.append((g, prs))
        for k in sorted(used):
            out.append(f"        m{k} = Ms[{blk[k] * MSTRIDE}];")
        for s in range(0, len(work), GROUP):
            grp = work[s:s + GROUP]
            for k, (g, _) in enumerate(grp):
                out.append(f"        d{k} = Dl[{g * 32}];")
            for k, (_, prs) in enumerate(grp):
                for ia, km in prs:
                    out.append(f"        L[{ia}] += d{k} * m{km};")
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
    lines += ["template <int P, int W>", "struct M2LWarp;", ""]
    for P in ORDERS:
        mb = MBLOCK[P]
        for w, aset in enumerate(warp_sets(P)):
            lines += [
                "template <>",
                f"struct M2LWarp<{P}, {w}> {{",
                f"    static constexpr int n = {len(aset)};",
                "    // the local-coefficient multi-indices this warp accumulates, in order",
                "    static __device__ __forceinline__ int alpha(int k)",
                "    {",
                f"        constexpr short a[{len(aset)}] = {{{', '.join(str(x) for x in aset)}}};",
                "        return a[k];",
                "    }",
                "    template <class R>",
                "    static __device__ __forceinline__ void run(const R* __restrict__ Dl, const R* __restrict__ Ms, R* L)",
                "    {",
                "        R " + ", ".join(f"m{i}" for i in range(mb)) + ";",
                "        R " + ", ".join(f"d{i}" for i in range(GROUP)) + ";",
            ]
            lines += body_blocked(P, mb, aset)
            lines += ["    }", "};", ""]
    print("\n".join(lines))


if __name__ == "__main__":
    main()
