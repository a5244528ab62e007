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
//   oracle_sort_par_{i32,f64,kv}   the same, with the two sides of large
//       ranges handed to separate threads (the paper's own suggestion of a
//       task-parallel recursion); bit-for-bit the sequential result.
//   oracle_select_{i32,f64}        k-th smallest key by repeated Appendix A
//       steps (quickselect); used to pick a true-median pivot.
//   oracle_mlp_*, oracle_bucket_*  the learned-splitter growth line (no
//       counterpart in the paper): the splitter MLP's forward pass and its loss
//       gradient in double precision, and the 256-way bucket partition by
//       splitters -- see the section at the end of this file.
//
// FP64 keys use IEEE '<' and '=='; inputs hold no NaN and no -0.0.
#include <cstdint>
#include <cmath>
#include <cstdlib>
#include <thread>

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
int quicksort_range(K *a, V &vals, int64_t first, int64_t last, double *trace, int64_t trace_cap, int64_t *ntrace)
{
    if (last <= first) return 0;
    int64_t cap = 64, size = 0;
    Range *stack = static_cast<Range *>(std::malloc(sizeof(Range) * cap));
    if (!stack) return -1;
    stack[size++] = Range{first, last};
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

template <class K, class V>
int quicksort(K *a, V &vals, int64_t n, double *trace, int64_t trace_cap, int64_t *ntrace)
{
    return quicksort_range(a, vals, int64_t(0), n - 1, trace, trace_cap, ntrace);
}

// The same Appendix A steps with the two sides of large ranges sorted by
// separate threads.  Every step touches only its own range, so the order in
// which disjoint ranges are processed cannot change the result: the output
// is bit-for-bit the sequential one (keys and values).
template <class K, class V>
int quicksort_parallel(K *a, V vals, int64_t left, int64_t right, int threads)
{
    if (threads <= 1 || right - left < (int64_t(1) << 16)) {
        V v = vals;
        return quicksort_range(a, v, left, right, nullptr, 0, nullptr);
    }
    int64_t lt_end, gt_begin;
    quicksort_step(a, vals, left, right, &lt_end, &gt_begin);
    int rc_low = 0;
    std::thread low([&] { rc_low = quicksort_parallel(a, vals, left, lt_end - 1, threads / 2); });
    const int rc_high = quicksort_parallel(a, vals, gt_begin, right, threads - threads / 2);
    low.join();
    return rc_low | rc_high;
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

int oracle_sort_par_i32(int32_t *a, int64_t n, int threads)
{
    return n < 2 ? 0 : quicksort_parallel(a, NoValues{}, int64_t(0), n - 1, threads);
}

int oracle_sort_par_f64(double *a, int64_t n, int threads)
{
    return n < 2 ? 0 : quicksort_parallel(a, NoValues{}, int64_t(0), n - 1, threads);
}

int oracle_sort_par_kv(int32_t *keys, int32_t *vals, int64_t n, int threads)
{
    return n < 2 ? 0 : quicksort_parallel(keys, Values{vals}, int64_t(0), n - 1, threads);
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

// ===========================================================================
// Learned splitters (growth line of the method; the paper has no model).
//
// Model: x (1024-key sorted sample, min-max scaled to [0,1]) -> h1 = relu(W1 x
// + b1) (64) -> h2 = relu(W2 h1 + b2) (64) -> z = W3 h2 + b3 (256) -> d =
// softplus(z) -> c = cumsum(d) -> q_j = c_j / c_255, j = 0..254: 255 monotone
// quantile estimates in (0, 1).  Loss = mean over the batch and j of
// (q_j - t_j)^2.  Parameters are one flat array in the order W1 (64x1024,
// row-major), b1, W2 (64x64), b2, W3 (256x64), b3.
// ===========================================================================
namespace {
constexpr int kIn = 1024, kHid = 64, kOut = 256, kSplit = 255;
constexpr long kOffW1 = 0, kOffB1 = kOffW1 + long(kHid) * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + long(kHid) * kHid,
               kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + long(kOut) * kHid, kNParams = kOffB3 + kOut;

double softplus(double z) { return z > 30.0 ? z : std::log1p(std::exp(z)); }
double sigmoid(double z) { return 1.0 / (1.0 + std::exp(-z)); }

struct Acts {
    double a1[kHid], h1[kHid], a2[kHid], h2[kHid], z[kOut], d[kOut], c[kOut], q[kSplit];
};

void forward_one(const double *p, const double *x, Acts &s)
{
    for (int o = 0; o < kHid; ++o) {
        double acc = p[kOffB1 + o];
        for (int i = 0; i < kIn; ++i) acc += p[kOffW1 + long(o) * kIn + i] * x[i];
        s.a1[o] = acc;
        s.h1[o] = acc > 0 ? acc : 0;
    }
    for (int o = 0; o < kHid; ++o) {
        double acc = p[kOffB2 + o];
        for (int i = 0; i < kHid; ++i) acc += p[kOffW2 + long(o) * kHid + i] * s.h1[i];
        s.a2[o] = acc;
        s.h2[o] = acc > 0 ? acc : 0;
    }
    double run = 0;
    for (int o = 0; o < kOut; ++o) {
        double acc = p[kOffB3 + o];
        for (int i = 0; i < kHid; ++i) acc += p[kOffW3 + long(o) * kHid + i] * s.h2[i];
        s.z[o] = acc;
        s.d[o] = softplus(acc);
        run += s.d[o];
        s.c[o] = run;
    }
    for (int j = 0; j < kSplit; ++j) s.q[j] = s.c[j] / s.c[kOut - 1];
}
}  // namespace

extern "C" {

long oracle_mlp_nparams(void) { return kNParams; }

// q[b*255 + j] for b < batch.
void oracle_mlp_forward(const double *params, const double *x, long batch, double *q)
{
    Acts s;
    for (long b = 0; b < batch; ++b) {
        forward_one(params, x + b * kIn, s);
        for (int j = 0; j < kSplit; ++j) q[b * kSplit + j] = s.q[j];
    }
}

// Loss (mean squared error over batch x 255) and its gradient with respect to
// every parameter, by the chain rule written out layer by layer.
double oracle_mlp_loss_grad(const double *params, const double *x, const double *t, long batch, double *grad)
{
    const double *p = params;
    for (long i = 0; i < kNParams; ++i) grad[i] = 0;
    double loss = 0;
    const double scale = 1.0 / (double(batch) * kSplit);
    Acts s;
    for (long b = 0; b < batch; ++b) {
        const double *xb = x + b * kIn;
        const double *tb = t + b * kSplit;
        forward_one(p, xb, s);
        double gq[kSplit];
        for (int j = 0; j < kSplit; ++j) {
            const double e = s.q[j] - tb[j];
            loss += e * e * scale;
            gq[j] = 2.0 * e * scale;
        }
        // q_j = c_j / S with S = c_255
        const double S = s.c[kOut - 1];
        double gc[kOut];
        double tail = 0;
        for (int j = 0; j < kSplit; ++j) {
            gc[j] = gq[j] / S;
            tail += gq[j] * s.c[j];
        }
        gc[kOut - 1] = -tail / (S * S);
        // c_k = sum_{i<=k} d_i  =>  gd_i = sum_{k>=i} gc_k
        double gd[kOut];
        double acc = 0;
        for (int i = kOut - 1; i >= 0; --i) {
            acc += gc[i];
            gd[i] = acc;
        }
        double gz[kOut];
        for (int i = 0; i < kOut; ++i) gz[i] = gd[i] * sigmoid(s.z[i]);
        double gh2[kHid] = {0};
        for (int o = 0; o < kOut; ++o) {
            grad[kOffB3 + o] += gz[o];
            for (int i = 0; i < kHid; ++i) {
                grad[kOffW3 + long(o) * kHid + i] += gz[o] * s.h2[i];
                gh2[i] += p[kOffW3 + long(o) * kHid + i] * gz[o];
            }
        }
        double ga2[kHid];
        for (int i = 0; i < kHid; ++i) ga2[i] = s.a2[i] > 0 ? gh2[i] : 0;
        double gh1[kHid] = {0};
        for (int o = 0; o < kHid; ++o) {
            grad[kOffB2 + o] += ga2[o];
            for (int i = 0; i < kHid; ++i) {
                grad[kOffW2 + long(o) * kHid + i] += ga2[o] * s.h1[i];
                gh1[i] += p[kOffW2 + long(o) * kHid + i] * ga2[o];
            }
        }
        for (int o = 0; o < kHid; ++o) {
            const double ga1 = s.a1[o] > 0 ? gh1[o] : 0;
            grad[kOffB1 + o] += ga1;
            for (int i = 0; i < kIn; ++i) grad[kOffW1 + long(o) * kIn + i] += ga1 * xb[i];
        }
    }
    return loss;
}

// 256-way bucket partition by sorted splitters (nsplit of them, non-decreasing):
// bucket(k) = number of splitters <= k.  out holds the buckets in order, each
// keeping input order; counts[b] = keys in bucket b (nsplit + 1 buckets).
}  // extern "C"

namespace {
template <class K>
void bucket_partition(const K *in, K *out, long n, const K *spl, int nsplit, int64_t *counts)
{
    for (int b = 0; b <= nsplit; ++b) counts[b] = 0;
    auto bucket = [&](K k) {
        int b = 0;
        while (b < nsplit && !(k < spl[b])) ++b;  // splitter <= key
        return b;
    };
    for (long i = 0; i < n; ++i) counts[bucket(in[i])]++;
    int64_t *pos = new int64_t[nsplit + 1];
    int64_t run = 0;
    for (int b = 0; b <= nsplit; ++b) {
        pos[b] = run;
        run += counts[b];
    }
    for (long i = 0; i < n; ++i) out[pos[bucket(in[i])]++] = in[i];
    delete[] pos;
}
}  // namespace

extern "C" {

void oracle_bucket_i32(const int32_t *in, int32_t *out, long n, const int32_t *spl, int nsplit, int64_t *counts)
{
    bucket_partition(in, out, n, spl, nsplit, counts);
}

void oracle_bucket_f64(const double *in, double *out, long n, const double *spl, int nsplit, int64_t *counts)
{
    bucket_partition(in, out, n, spl, nsplit, counts);
}

}  // extern "C"

extern "C" {

// One Adam step (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
void oracle_adam_step(double *p, const double *g, double *m, double *v, long n, long step, double lr, double b1,
                      double b2, double eps)
{
    const double c1 = 1.0 - std::pow(b1, double(step)), c2 = 1.0 - std::pow(b2, double(step));
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
    }
}

}  // extern "C"
