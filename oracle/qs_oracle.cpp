// Oracle for the hybrid Quicksort hot path -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously correct CPU statement of what the CUDA path
// computes.  Only the tests, the package's smoke check and the benchmark's
// CPU-baseline leg may load this file; the product path never does.  It shares
// no code, header, table or helper with the CUDA sources, and uses no library
// algorithm: every comparison and move is written out below.
//
//   oracle_partition_{i32,f64,kv}  Section III-B (partitioning).  Keys strictly
//       below the pivot go first, keys at-or-above it last; the return value
//       is the split index = number of keys below the pivot (the paper's
//       'left_w').  The paper leaves the order inside each side open; this
//       oracle fixes the order a one-pass scan produces: the lower side in
//       input order, the upper side in REVERSE input order (it is filled from
//       the end of the array, like the paper's right_w iterator).
//   oracle_sort_{i32,f64,kv}       Appendix A scalar Quicksort: middle pivot
//       swapped to the end, one forward sweep moving keys strictly below the
//       pivot to the front, pivot swapped into the bound, recurse on both
//       sides.  Two readings where the paper is silent:
//         (1) the recursion is an explicit stack, smaller side first, so 2^30
//             keys cannot overflow the call stack;
//         (2) after the pivot is placed, keys equal to it are gathered next to
//             it and take no further part (Appendix A alone is quadratic on
//             all-equal input, e.g. the few-unique workloads).
//       Key/value sorting (Section III-D) applies every key move to the value
//       array too.
//   oracle_select_{i32,f64}        k-th smallest key by repeated Appendix A
//       steps (quickselect); used to pick a true-median pivot.
//
// FP64 keys use IEEE '<' and '=='; inputs hold no NaN and no -0.0.
#include <cstdint>
#include <cstdlib>

namespace {

// Values ride along with keys (Section III-D) or are absent.
struct NoValues {
    void swap(int64_t, int64_t) {}
};
struct Values {
    int32_t *v;
    void swap(int64_t i, int64_t j)
    {
        int32_t t = v[i];
        v[i] = v[j];
        v[j] = t;
    }
};

template <class K, class V>
void swap_pair(K *a, V &vals, int64_t i, int64_t j)
{
    K t = a[i];
    a[i] = a[j];
    a[j] = t;
    vals.swap(i, j);
}

// Section III-B partition with the canonical order described above.
template <class K>
int64_t partition_copy(const K *in, const int32_t *vin, K *out, int32_t *vout, int64_t n, K pivot)
{
    int64_t lo = 0, hi = n;
    for (int64_t i = 0; i < n; ++i) {
        if (in[i] < pivot) {
            out[lo] = in[i];
            if (vin) vout[lo] = vin[i];
            ++lo;
        } else {
            --hi;
            out[hi] = in[i];
            if (vin) vout[hi] = vin[i];
        }
    }
    return lo;
}

// Appendix A 'partition': sweep idx = left..right, moving keys strictly below
// the pivot value to the front; returns the bound.
template <class K, class V>
int64_t appendix_partition(K *a, V &vals, int64_t left, int64_t right, K pivot)
{
    for (int64_t idx = left; idx <= right; ++idx) {
        if (a[idx] < pivot) {
            swap_pair(a, vals, idx, left);
            ++left;
        }
    }
    return left;
}

// One Appendix A step on a[left..right] (left < right) plus reading (2).
// Afterwards a[left..lt_end) < pivot, a[lt_end..gt_begin) == pivot and
// a[gt_begin..right] > pivot.  Returns the pivot value.
template <class K, class V>
K quicksort_step(K *a, V &vals, int64_t left, int64_t right, int64_t *lt_end, int64_t *gt_begin)
{
    int64_t pivot_idx = (right - left) / 2 + left;  // naive middle pick
    swap_pair(a, vals, pivot_idx, right);
    K pivot = a[right];
    int64_t bound = appendix_partition(a, vals, left, right, pivot);
    swap_pair(a, vals, bound, right);
    // Reading (2): gather keys equal to the pivot right after it.
    int64_t eq_end = bound + 1;
    for (int64_t idx = bound + 1; idx <= right; ++idx) {
        if (a[idx] == pivot) {
            swap_pair(a, vals, idx, eq_end);
            ++eq_end;
        }
    }
    *lt_end = bound;
    *gt_begin = eq_end;
    return pivot;
}

struct Range {
    int64_t left, right;
};

// Appendix A 'QS_core' with the explicit stack of reading (1).  Optionally
// records each chosen pivot (in the order chosen).  Returns 0, or -1 when the
// stack cannot grow.
template <class K, class V>
int quicksort(K *a, V &vals, int64_t n, double *trace, int64_t trace_cap, int64_t *ntrace)
{
    if (n < 2) return 0;
    int64_t cap = 64, size = 0;
    Range *stack = static_cast<Range *>(std::malloc(sizeof(Range) * cap));
    if (!stack) return -1;
    stack[size++] = Range{0, n - 1};
    while (size > 0) {
        Range r = stack[--size];
        int64_t left = r.left, right = r.right;
        while (left < right) {
            int64_t lt_end, gt_begin;
            K pivot = quicksort_step(a, vals, left, right, &lt_end, &gt_begin);
            if (ntrace) {
                if (*ntrace < trace_cap) trace[*ntrace] = static_cast<double>(pivot);
                ++*ntrace;
            }
            int64_t n_low = lt_end - left, n_high = right - gt_begin + 1;
            Range larger = n_low < n_high ? Range{gt_begin, right} : Range{left, lt_end - 1};
            if (larger.right > larger.left) {
                if (size == cap) {
                    cap *= 2;
                    Range *p = static_cast<Range *>(std::realloc(stack, sizeof(Range) * cap));
                    if (!p) {
                        std::free(stack);
                        return -1;
                    }
                    stack = p;
                }
                stack[size++] = larger;
            }
            if (n_low < n_high) {
                right = lt_end - 1;
            } else {
                left = gt_begin;
            }
        }
    }
    std::free(stack);
    return 0;
}

template <class K>
K select_kth(K *a, int64_t n, int64_t k)
{
    NoValues none;
    int64_t left = 0, right = n - 1;
    while (left < right) {
        int64_t lt_end, gt_begin;
        K pivot = quicksort_step(a, none, left, right, &lt_end, &gt_begin);
        if (k < lt_end)
            right = lt_end - 1;
        else if (k >= gt_begin)
            left = gt_begin;
        else
            return pivot;
    }
    return a[k];
}

}  // namespace

extern "C" {

int64_t oracle_partition_i32(const int32_t *in, int32_t *out, int64_t n, int32_t pivot)
{
    return partition_copy<int32_t>(in, nullptr, out, nullptr, n, pivot);
}

int64_t oracle_partition_f64(const double *in, double *out, int64_t n, double pivot)
{
    return partition_copy<double>(in, nullptr, out, nullptr, n, pivot);
}

int64_t oracle_partition_kv(const int32_t *kin, const int32_t *vin, int32_t *kout, int32_t *vout,
                            int64_t n, int32_t pivot)
{
    return partition_copy<int32_t>(kin, vin, kout, vout, n, pivot);
}

int oracle_sort_i32(int32_t *a, int64_t n)
{
    NoValues none;
    return quicksort(a, none, n, nullptr, 0, nullptr);
}

int oracle_sort_f64(double *a, int64_t n)
{
    NoValues none;
    return quicksort(a, none, n, nullptr, 0, nullptr);
}

int oracle_sort_kv(int32_t *keys, int32_t *vals, int64_t n)
{
    Values v{vals};
    return quicksort(keys, v, n, nullptr, 0, nullptr);
}

int oracle_sort_trace_i32(int32_t *a, int64_t n, double *trace, int64_t trace_cap, int64_t *ntrace)
{
    NoValues none;
    *ntrace = 0;
    return quicksort(a, none, n, trace, trace_cap, ntrace);
}

int32_t oracle_select_i32(int32_t *a, int64_t n, int64_t k) { return select_kth(a, n, k); }

double oracle_select_f64(double *a, int64_t n, int64_t k) { return select_kth(a, n, k); }

}  // extern "C"
