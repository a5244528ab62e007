// Leaf sort of a part held by a group of threads: Bitonic runs in registers,
// merged by merge path in shared memory.
//
// Every thread first sorts its E keys in registers with the paper's Bitonic
// network (Section III-A, Algorithms 1-2: the flip form, every comparator
// putting the minimum at the lower index), and groups of 2 and then 4 lanes
// continue the same network across lanes with shuffles (the paper's
// multi-vector sort, the permutation across vectors becoming
// __shfl_xor_sync), which gives sorted runs of 4E keys.  The group then
// merges the runs pairwise -- 4E, 8E, 16E, ... -- until one run holds the
// whole part.  In a merge level every thread produces E consecutive outputs:
// it finds where its first output comes from with a binary search along its
// diagonal of the merge grid ("merge path"), then takes E keys from the two
// runs' heads, one comparison each.
//
// Why not the Bitonic network all the way up: a Bitonic merge of two runs of
// m keys costs log2(2m) compare-exchange stages per key, a merge-path merge
// one comparison per key, so above a few runs the merge is cheaper; both are
// bound by integer ALU work on this GPU.  The merge needs no power-of-two
// padding either: a part is padded to a multiple of 32*E keys only.
//
// Layout trick (the Bitonic sequence again): in shared memory every run that
// will be the right-hand operand of its merge is stored reversed, so the two
// runs of a merge form an ascending-then-descending sequence.  When one run
// is exhausted, its read pointer walks on into the other run from that run's
// largest end: such a key is never smaller than the other run's head unless
// every remaining key is equal, so it serves as a sentinel and the merge loop
// needs no bounds checks.
//
// Ties: equal sort-space words are bit-identical (key/value pairs are packed
// into one word), so which copy a merge emits first is irrelevant.  The
// padding is the largest sort-space word; it ends at the tail like in the
// paper's wrapper (Section III-A-3).
#pragma once

#include "qs_bitonic.cuh"

namespace qs {

// Shared-memory slot of element w of a group's slice.  A row of E elements
// is one thread's run (128 bytes for both key widths: E = 16 words of 8
// bytes, or 32 of 4); the position inside a row is XORed with the row
// number, so a thread storing its run (one element per row across a warp)
// and a warp reading consecutive elements both hit distinct banks.
template <int E>
__device__ __forceinline__ int swz(int w)
{
    static_assert(E == 16 || E == 32, "one 128-byte row per thread");
    constexpr int LE = E == 16 ? 4 : 5;
    const unsigned u = static_cast<unsigned>(w);  // w >= 0: shifts, no signed division
    return static_cast<int>(u ^ ((u >> LE) & (E - 1)));
}

// Sorts the ng*E elements of a group of ng threads (ng a multiple of 32, the
// group starting at a multiple of 32 threads); thread g of the group holds E
// of them in k on entry, in any order.  On exit the sorted elements are in
// sm (slots swz(0 .. ng*E-1), ascending).
template <int E, class S>
__device__ void group_merge_sort(S (&k)[E], S *sm, int g, int ng, int bar)
{
    const int P = ng * E;
    const int lane = g & 31;
    // Runs of E (registers), 2E and 4E (lanes).  (Running the warp network
    // on up to 32E keys instead measured slower: its shuffle stages with
    // run-time lane masks cost more per key than merge-path levels.)
    reg_merges<E, 2, S>(k);
    shfl_flip<E, S>(k, 1, (lane & 1) != 0);
    reg_half<E, E / 2>(k);
    shfl_flip<E, S>(k, 3, (lane & 2) != 0);
    shfl_half<E, S>(k, 1, (lane & 1) != 0);
    reg_half<E, E / 2>(k);
    {
        // Run j = g/4 holds [4E*j, 4E*j + 4E); odd runs are stored reversed.
        const int q0 = g * E;
        const int run0 = q0 & ~(4 * E - 1);
        const bool rev = (g >> 2) & 1;
        const int base = rev ? run0 + 4 * E - 1 - (q0 - run0) : q0;
        const int step = rev ? -1 : 1;
#pragma unroll
        for (int r = 0; r < E; ++r) sm[swz<E>(base + step * r)] = k[r];
    }
    for (int W = 4 * E; W < P; W <<= 1) {
        // A merge level reads and writes only its pair's slots [pa, pa + 2W),
        // which the previous level's threads of the same pair wrote: while a
        // pair spans at most 32 runs, those threads are one warp (pairs are
        // aligned to their width), and the warp alone synchronises.
        const bool in_warp = 2 * W <= 32 * E;
        if (in_warp)
            __syncwarp();
        else
            group_sync(bar, ng);
        const int o0 = g * E;
        const int pa = o0 & ~(2 * W - 1);
        const int na = P - pa < W ? P - pa : W;
        const int pb = pa + na;
        const int nb = P - pb < W ? (P - pb > 0 ? P - pb : 0) : W;
        const int d = o0 - pa;
        // Merge path: i = elements of A among the first d outputs.  A[x] is
        // slot pa + x, B[y] (reversed) slot pb + nb - 1 - y, so B[d-1-mid]
        // is slot cb + mid.
        const int cb = pb + nb - d;
        int lo = d > nb ? d - nb : 0;
        int hi = d < na ? d : na;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sm[swz<E>(pa + mid)] <= sm[swz<E>(cb + mid)])
                lo = mid + 1;
            else
                hi = mid;
        }
        int ia = pa + lo;                 // next A slot (forward)
        int ib = pb + nb - 1 - (d - lo);  // next B slot (backward)
        S a = sm[swz<E>(ia)];
        S b = sm[swz<E>(ib)];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const bool ta = a <= b;
            k[r] = ta ? a : b;
            if (r + 1 < E) {
                ia += ta ? 1 : 0;
                ib -= ta ? 0 : 1;
                const S nx = sm[swz<E>(ta ? ia : ib)];
                a = ta ? nx : a;
                b = ta ? b : nx;
            }
        }
        // The output run (2W wide, the last one possibly shorter) is stored
        // reversed if it will be a right-hand operand of the next level.
        const bool rev = (pa & (2 * W)) != 0;  // pa is a multiple of 2W: the output run's parity
        const int base = rev ? pa + na + nb - 1 - d : o0;
        const int step = rev ? -1 : 1;
        if (in_warp)
            __syncwarp();
        else
            group_sync(bar, ng);
#pragma unroll
        for (int r = 0; r < E; ++r) sm[swz<E>(base + step * r)] = k[r];
    }
}

}  // namespace qs
