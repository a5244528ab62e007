// Leaf sort of a part held by a group of threads: Bitonic runs in registers,
// merged by merge path in shared memory.
//
// Every thread first sorts its E keys in registers with the paper's Bitonic
// network (Section III-A, Algorithms 1-2: the flip form, every comparator
// putting the minimum at the lower index; reg_merges below).  The group then
// merges the sorted runs pairwise -- runs of E, 2E, 4E, ... keys -- until one
// run holds the whole part.  In a merge level every thread produces E
// consecutive outputs: it finds where its first output comes from with a
// binary search along its diagonal of the merge grid ("merge path"), then
// takes E keys from the two runs' heads, one comparison each.
//
// Why not the Bitonic network all the way up: a Bitonic merge of two runs of
// m keys costs log2(2m) compare-exchange stages per key, a merge-path merge
// one comparison per key, so sorting P keys costs E-run networks plus
// log2(P/E) merge levels instead of log2(P)(log2(P)+1)/2 network stages; on
// this GPU both are bound by integer ALU work, so the cheaper one wins (and
// it needs no power-of-two padding: a part is padded to a multiple of 32*E
// keys only).
//
// Ties: the merge takes the left run's key first, so equal keys never cross;
// equal sort-space words are bit-identical (key/value pairs are packed into
// one word), so the order among them is irrelevant anyway.  The padding is
// the largest sort-space word; it ends at the tail like in the paper's
// wrapper (Section III-A-3).
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
    return w ^ ((w / E) & (E - 1));
}

// Number of elements of run A (at a0, na long) among the first d outputs of
// the merge of A and B (at b0, nb long), taking A's element first on ties.
template <int E, class S>
__device__ __forceinline__ int merge_path(const S *sm, int a0, int na, int b0, int nb, int d)
{
    int lo = d > nb ? d - nb : 0;
    int hi = d < na ? d : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sm[swz<E>(a0 + mid)] <= sm[swz<E>(b0 + d - 1 - mid)])
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Sorts the ng*E elements of a group of ng threads (ng a multiple of 32);
// thread g of the group holds E of them in k on entry (any distribution).
// On exit the sorted elements are in sm (slots swz(0 .. ng*E-1)), and thread
// g's registers hold elements g*E .. g*E+E-1.  `big` is the largest
// sort-space word (the padding and the exhausted-run sentinel).
template <int E, class S>
__device__ void group_merge_sort(S (&k)[E], S *sm, int g, int ng, int bar, S big)
{
    const int P = ng * E;
    reg_merges<E, 2, S>(k);
#pragma unroll
    for (int r = 0; r < E; ++r) sm[swz<E>(g * E + r)] = k[r];
    for (int W = E; W < P; W <<= 1) {
        group_sync(bar, ng);
        const int o0 = g * E;
        const int pa = o0 & ~(2 * W - 1);
        const int na = P - pa < W ? P - pa : W;
        const int pb = pa + na;
        const int nb = P - pb < W ? (P - pb > 0 ? P - pb : 0) : W;
        const int d = o0 - pa;
        const int i = merge_path<E, S>(sm, pa, na, pb, nb, d);
        int ia = pa + i, ib = pb + d - i;
        const int ea = pa + na, eb = pb + nb;
        S a = ia < ea ? sm[swz<E>(ia)] : big;
        S b = ib < eb ? sm[swz<E>(ib)] : big;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            // An exhausted run shows `big`: taking it instead of a real `big`
            // key of the other run emits the same word.
            const bool ta = a <= b;
            k[r] = ta ? a : b;
            if (r + 1 < E) {
                ia += ta ? 1 : 0;
                ib += ta ? 0 : 1;
                const int p = ta ? ia : ib;
                const int e = ta ? ea : eb;
                const S nx = p < e ? sm[swz<E>(p)] : big;
                a = ta ? nx : a;
                b = ta ? b : nx;
            }
        }
        group_sync(bar, ng);
#pragma unroll
        for (int r = 0; r < E; ++r) sm[swz<E>(o0 + r)] = k[r];
    }
}

}  // namespace qs
