// Theta join after Algorithm 3 (Sec. 4.2), on one GPU.
//
// Both tables are cut into ranges ("groups") of one column with the same
// boundaries for R and S (equal-width, power-of-two wide, from the minimum
// over both tables), by a one-pass range partition.  A pair of groups
// (x = R group, y = S group) is a region of the paper's matrix:
//   - band >= 0 (predicate (R.a op S.a) AND |R.k - S.k| <= band, groups on k):
//     only regions with |x - y| <= ceil(band / width) can hold results.  For
//     each S group y the R rows of those groups are contiguous after the
//     partition (the "window"); they are staged in shared memory, sorted
//     into fine k-buckets, and each S row scans only the buckets that
//     intersect [k - band, k + band] before testing both conjuncts exactly.
//   - band < 0 (predicate R.a op S.a, groups on a): the diagonal region
//     (x == y) is compared pair by pair (the paper's GPU_theta_join);
//     regions whose ranges already decide the predicate (x < y for <, <=;
//     x > y for >, >=; x != y for != and ANY) are written as cross products
//     without any comparison; the others are skipped.
// Each work item is (S group, R chunk, S chunk).  Count pass -> scan ->
// one exact allocation -> emit pass, as in the other joins.
#include "jn_algos.h"
#include "jn_partition.cuh"

namespace jnx {

constexpr int TH_T = 256;
#ifndef JN_TH_RCAP
#define JN_TH_RCAP 4096
#endif
constexpr int TH_RCAP = JN_TH_RCAP;   // R rows per shared-memory chunk
constexpr int TH_SCH = 4096;    // S rows per work item
constexpr int TH_KPAD = 4;      // staged rows of padding read by the unrolled candidate scan
constexpr int TH_NFB = 2048;    // fine k-buckets per window
constexpr uint64_t CE_CHUNK = 1u << 16;  // cross-product pairs per work item

// Dynamic shared memory of the theta join kernel: the staged R rows (k and a,
// then payloads) and the fine-bucket offsets.
template <typename K>
static size_t theta_smem(int) {
    return (size_t)(TH_RCAP + TH_KPAD) * 2 * sizeof(K) + (size_t)TH_RCAP * 4 + sizeof(uint32_t) * TH_NFB;
}

// Minimum and maximum of a column into mm[0], mm[1] (atomics, one per block).
// The body is read in 16-byte words, four in flight per thread; the elements
// before the first 16-byte boundary and after the last whole word are read
// one by one.
template <typename K>
__global__ void __launch_bounds__(512) k_minmax(const K* __restrict__ col, int64_t n, long long* __restrict__ mm) {
    constexpr int PER = 16 / sizeof(K);
    __shared__ long long s_lo[16], s_hi[16];
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    auto take = [&](long long v) {
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    };
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t head = min(n, (int64_t)(((16 - ((uintptr_t)col & 15)) & 15) / sizeof(K)));
    const int64_t nv = (n - head) / PER;
    if (tid < head) take((long long)col[tid]);
    const uint4* v = reinterpret_cast<const uint4*>(col + head);
#pragma unroll 4
    for (int64_t i = tid; i < nv; i += stride) {
        const uint4 w = __ldg(v + i);
        if (sizeof(K) == 4) {
            take((int32_t)w.x);
            take((int32_t)w.y);
            take((int32_t)w.z);
            take((int32_t)w.w);
        } else {
            take((long long)(((uint64_t)w.y << 32) | w.x));
            take((long long)(((uint64_t)w.w << 32) | w.z));
        }
    }
    for (int64_t i = head + nv * PER + tid; i < n; i += stride) take((long long)col[i]);
    // minima combine with minima and maxima with maxima: a thread without
    // elements holds the empty range (LLONG_MAX, LLONG_MIN)
    auto merge = [&](long long l, long long h) {
        lo = l < lo ? l : lo;
        hi = h > hi ? h : hi;
    };
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        merge(__shfl_xor_sync(0xffffffffu, lo, o), __shfl_xor_sync(0xffffffffu, hi, o));
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_lo[w] = lo;
        s_hi[w] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) merge(s_lo[k], s_hi[k]);
        if (lo <= hi) {
            atomicMin(&mm[0], lo);
            atomicMax(&mm[1], hi);
        }
    }
}

__global__ void k_mm_init(long long* mm) {
    mm[0] = LLONG_MAX;
    mm[1] = LLONG_MIN;
}

// Group width 2^shift: the smallest power of two with (hi - lo) >> shift < G.
__global__ void k_range_setup(const long long* __restrict__ mm, int G, RangeParams* __restrict__ p) {
    long long lo = mm[0], hi = mm[1];
    if (lo > hi) { lo = 0; hi = 0; }  // both tables empty in this column
    const uint64_t span = (uint64_t)hi - (uint64_t)lo;
    int s = 0;
    while (s < 63 && (span >> s) >= (uint64_t)G) s++;
    p->lo = lo;
    p->hi = hi;
    p->shift = s;
    p->groups = (int)(span >> s) + 1;
    p->fshift = 0;
    p->pad = 0;
}

// Offset of value k from lo (k must lie in [lo, hi]).
template <typename K>
__device__ __forceinline__ uint64_t uoff(K k, long long lo) {
    return (uint64_t)(long long)k - (uint64_t)lo;
}

// Window of S group y in offset space: [y*w - band, (y+1)*w - 1 + band] ∩ [0, span].
__device__ __forceinline__ void window_of(const RangeParams& p, int y, long long band, uint64_t* wlo,
                                          uint64_t* whi) {
    const uint64_t span = (uint64_t)p.hi - (uint64_t)p.lo;
    const uint64_t g0 = (uint64_t)y << p.shift;
    const uint64_t g1 = ((uint64_t)(y + 1) << p.shift) - 1;
    const uint64_t b = band < 0 ? 0 : (uint64_t)band;
    *wlo = g0 > b ? g0 - b : 0;
    *whi = (b > span || g1 + b > span || g1 + b < g1) ? span : g1 + b;
}

// Number of neighbouring groups a band reaches: ceil(band / width).
__device__ __forceinline__ int band_groups(const RangeParams& p, long long band, int G) {
    if (band <= 0) return 0;
    const uint64_t w = (uint64_t)1 << p.shift;
    const uint64_t d = ((uint64_t)band + w - 1) >> p.shift;
    return d > (uint64_t)G ? G : (int)d;
}

// Joins of one launch: join i owns partitions [i << lg, (i + 1) << lg) (its
// groups y = p & (2^lg - 1), of which the first groups[i] are in use) and has
// its own range parameters, band and op.  A single join is the case of one.
struct ThetaSet {
    const RangeParams* prm;
    const long long* band;
    const int* op;
    const int* groups;
    int lg;
};

__global__ void k_set_theta_one(long long* band, int* op, int* groups, long long b, int o, int g) {
    *band = b;
    *op = o;
    *groups = g;
}

// items[p] = R chunks of the window of group y of its join x S chunks of y.
// With `bound`, adds sum_y |window of y| * |S_y| to it: the pairs the
// compared regions hold (Eq. (rsize)'s allocation for them).
__global__ void k_theta_items(const uint64_t* __restrict__ roff, const uint64_t* __restrict__ soff, ThetaSet ts,
                              int P, uint64_t* __restrict__ items, unsigned long long* __restrict__ bound) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t nrw = 0, ns = 0;
    if (p < P) {
        const int inst = p >> ts.lg, y = p & ((1 << ts.lg) - 1), G = ts.groups[inst];
        if (y < G) {
            const int dg = band_groups(ts.prm[inst], ts.band[inst], G);
            const int base = inst << ts.lg;
            const int x0 = base + max(0, y - dg), x1 = base + min(G - 1, y + dg);
            nrw = roff[x1 + 1] - roff[x0];
            ns = soff[p + 1] - soff[p];
        }
        items[p] = (nrw && ns) ? ((nrw + TH_RCAP - 1) / TH_RCAP) * ((ns + TH_SCH - 1) / TH_SCH) : 0;
    }
    if (bound) warp_add_to(bound, nrw * ns);  // < |R| * |S| < 2^62: no overflow
}

// BAND: window + fine buckets; !BAND: diagonal group, every pair compared.
// ka = compared column (a), kk = grouped column (k; equals ka when !BAND).
// Rows: key = the grouped column (k for a band, a otherwise), b = column a
// (band only), pay = payload.
template <typename K, bool BAND>
__device__ __forceinline__ K col_a(const Row<K, BAND>& x) {
    if constexpr (BAND) return x.b; else return x.key;
}

// One staged R row of a theta work item: its grouped column k and column a.
template <typename K>
struct alignas(2 * sizeof(K)) KA {
    K k;
    K a;
};

// Writes (R payload, spay) to out[0 ..) for every staged R row in [lo, hi)
// that passes one S row's intervals.  PLAIN: the a-interval is not inverted,
// so the test is the bare range check; a band interval is never inverted.
template <bool PLAIN, typename K, bool BAND>
__device__ __forceinline__ void theta_emit_scan(const KA<K>* s_ka, const int32_t* s_p, uint32_t lo, uint32_t hi,
                                                const Interval<K>& ia, const Interval<K>& ib, jn_pair* out,
                                                int32_t spay) {
    for (uint32_t e = lo; e < hi; e++) {
        const KA<K> t = s_ka[e];
        bool ok = PLAIN ? in_range(t.a, ia.lo, ia.span) : iv_test(ia, t.a);
        if (BAND) ok &= in_range(t.k, ib.lo, ib.span);
        if (ok) {
            st_pair(out++, s_p[e], spay);
        }
    }
}

// Tests one S row against the staged candidates [lo, hi), four shared loads
// in flight (the loads past hi read the padding behind the staged rows and
// are discarded).  Returns the matches; *mask gets the matches among the
// first 32 candidates as bits, *fsum (AGG) the sum of f over the matches.
// PLAIN: the a-interval is not inverted, so its test is the bare range check.
template <bool PLAIN, bool AGG, typename K, bool BAND>
__device__ __forceinline__ uint32_t theta_scan(const KA<K>* s_ka, const int32_t* s_p, uint32_t lo, uint32_t hi,
                                               const Interval<K>& ia, const Interval<K>& ib, uint32_t* mask,
                                               unsigned long long* fsum) {
    uint32_t m = 0, mk = 0, bit = 1;
    for (uint32_t e = lo; e < hi; e += 4) {
        KA<K> t[4];
#pragma unroll
        for (int u = 0; u < 4; u++) t[u] = s_ka[e + u];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            bool ok = PLAIN ? in_range(t[u].a, ia.lo, ia.span) : iv_test(ia, t[u].a);
            if (BAND) ok &= in_range(t[u].k, ib.lo, ib.span);
            ok &= e + u < hi;
            m += ok;
            mk |= ok ? bit : 0u;
            bit <<= 1;
            if (AGG && ok) *fsum += chk_f(s_p[e + u]);
        }
    }
    *mask = mk;
    return m;
}

// What the count pass of a band join leaves for a gathering emit pass.  For
// S row j of item it, rows[it * TH_SCH + j] = (mask, at): the row's matches
// among its first 32 candidates as bits, and at = (offset of its first pair
// within the item's output << 13) | (staged position of its first candidate),
// or TH_WIDE when the row has more than 32 candidates.  pay[it * TH_RCAP ..]
// holds the item's staged R payloads in staged order.  sdesc[it] =
// (first S row << 14) | (S rows << 1) | wide, wide when any of its rows is;
// *any_wide is set when some item is wide.  Wide items are emitted by the
// join kernel itself, the others by k_theta_gather.
struct ThetaRec {
    uint2* rows;
    int32_t* pay;
    uint64_t* sdesc;
    unsigned int* any_wide;
};
constexpr uint32_t TH_WIDE = 0xFFFFFFFFu;
static_assert(TH_SCH == 4096 && TH_RCAP < 8192, "record fields: 12 bits of S row, 13 of staged position");

constexpr int TH_GSTG = 256;  // pairs a gather warp stages before one coalesced store

// Emit pass of the band items that are not wide, one block per item: the
// item's staged payloads are loaded into shared memory, and each warp takes
// the 32 S rows one warp of the count pass took (same rows per round and
// warp), whose pairs are one contiguous run of the output.  The warp gathers
// the run from the rows' records into shared memory and stores it coalesced
// (a run longer than TH_GSTG pairs is written lane by lane).
template <typename K>
__global__ void __launch_bounds__(TH_T)
k_theta_gather(const Row<K, true>* __restrict__ srows, const uint64_t* __restrict__ nitems_p,
               const uint64_t* __restrict__ item_off, ThetaRec rec, jn_pair* __restrict__ out) {
    __shared__ __align__(16) int32_t s_pay[TH_RCAP];
    __shared__ __align__(16) int2 s_stg[TH_T / 32][TH_GSTG];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t nitems = *nitems_p;
    for (uint64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const uint64_t d = rec.sdesc[it];
        if (d & 1) continue;  // wide: the join kernel emits it
        const int sn = (int)((d >> 1) & 8191);
        const uint64_t sbeg = d >> 14;
        __syncthreads();  // the previous item's payloads are no longer read
        const int4* src = reinterpret_cast<const int4*>(rec.pay + it * TH_RCAP);
        for (int i = threadIdx.x; i < TH_RCAP / 4; i += TH_T) reinterpret_cast<int4*>(s_pay)[i] = src[i];
        __syncthreads();
        const uint64_t obase = item_off[it];
        // a row's record and S payload load one round ahead of their use
        uint2 rn = make_uint2(0u, 0u);
        int32_t pn = 0;
        if ((int)threadIdx.x < sn) {
            rn = rec.rows[it * TH_SCH + threadIdx.x];
            pn = srows[sbeg + threadIdx.x].pay;
        }
        for (int r0 = 0; r0 < sn; r0 += TH_T) {
            const int j = r0 + threadIdx.x;
            uint32_t mask = rn.x;
            const uint32_t at = rn.y;
            const int32_t spay = pn;
            if (j + TH_T < sn) {
                rn = rec.rows[it * TH_SCH + j + TH_T];
                pn = srows[sbeg + j + TH_T].pay;
            } else {
                rn = make_uint2(0u, 0u);
            }
            const uint32_t m = __popc(mask);
            const uint32_t incl = warp_incl_scan(m);
            const uint32_t wt = __shfl_sync(0xffffffffu, incl, 31);
            if (wt == 0) continue;  // lane 0 holds a row whenever the warp has pairs
            const uint32_t run = __shfl_sync(0xffffffffu, (at >> 13) - (incl - m), 0);
            jn_pair* g = out + obase + run;
            const int32_t* rp = s_pay + (at & 8191);
            if (wt <= (uint32_t)TH_GSTG) {
                uint32_t q = incl - m;
                while (mask) {
                    const int e = __ffs(mask) - 1;
                    mask &= mask - 1;
                    s_stg[w][q++] = make_int2(rp[e], spay);
                }
                __syncwarp();
                for (uint32_t q2 = lane; q2 < wt; q2 += 32) st_pair(g + q2, s_stg[w][q2].x, s_stg[w][q2].y);
                __syncwarp();
            } else {
                jn_pair* o = g + (incl - m);
                while (mask) {
                    const int e = __ffs(mask) - 1;
                    mask &= mask - 1;
                    st_pair(o++, rp[e], spay);
                }
            }
        }
    }
}

template <typename K, int MODE, bool BAND>
__global__ void __launch_bounds__(TH_T)
k_theta_join(const Row<K, BAND>* __restrict__ rrows, const uint64_t* __restrict__ roff,
             const Row<K, BAND>* __restrict__ srows, const uint64_t* __restrict__ soff, ThetaSet ts, int Ptot,
             const uint64_t* __restrict__ item_prefix, unsigned long long* __restrict__ item_val,
             unsigned long long* __restrict__ chk, const uint64_t* __restrict__ item_off, jn_pair* __restrict__ out,
             unsigned int* __restrict__ work, ThetaRec rec) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the staged R rows' k and a side by side, so one load gives both
    KA<K>* s_ka = reinterpret_cast<KA<K>*>(smem);
    int32_t* s_p = reinterpret_cast<int32_t*>(s_ka + TH_RCAP + TH_KPAD);
    uint32_t* s_off = reinterpret_cast<uint32_t*>(s_p + TH_RCAP);
    __shared__ unsigned long long tmp64[33];
    __shared__ uint32_t tmp32[33];
    __shared__ unsigned int s_item;
    __shared__ uint32_t s_cursor, s_rows, s_wide;

    const uint64_t nitems = item_prefix[Ptot];
    const int lane = threadIdx.x & 31;
    // count pass of a band join followed by a gathering emit: record the rows
    const bool record = BAND && MODE == MODE_COUNT && rec.rows != nullptr;
    while (true) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(work, 1u);
            s_cursor = 0;
            s_rows = 0;
            s_wide = 0;
        }
        __syncthreads();
        const uint64_t it = s_item;
        if (it >= nitems) break;
        if (MODE == MODE_EMIT && rec.sdesc != nullptr && !(rec.sdesc[it] & 1)) {
            __syncthreads();  // a gathered item: k_theta_gather writes its pairs
            continue;
        }
        const int p = find_segment(item_prefix, Ptot, it);
        const int inst = p >> ts.lg, y = p & ((1 << ts.lg) - 1), G = ts.groups[inst];
        const RangeParams P = ts.prm[inst];
        const long long band = ts.band[inst];
        const int op = ts.op[inst];
        const int dg = BAND ? band_groups(P, band, G) : 0;
        const int gbase = inst << ts.lg;
        const int x0 = gbase + max(0, y - dg), x1 = gbase + min(G - 1, y + dg);
        const uint64_t wbeg = roff[x0], nrw = roff[x1 + 1] - wbeg;
        const uint64_t ns = soff[p + 1] - soff[p];
        const uint64_t nrc = (nrw + TH_RCAP - 1) / TH_RCAP;
        const uint64_t local = it - item_prefix[p];
        const uint64_t rc = local % nrc, sc = local / nrc;
        const uint64_t rbeg = wbeg + rc * TH_RCAP;
        const int rn = (int)min((uint64_t)TH_RCAP, nrw - rc * TH_RCAP);
        const uint64_t sbeg = soff[p] + sc * TH_SCH;
        const int sn = (int)min((uint64_t)TH_SCH, ns - sc * TH_SCH);

        uint64_t wlo = 0, whi = 0;
        int fs = 0, nfb = 1;
        if (BAND) {
            window_of(P, y, band, &wlo, &whi);
            while (((whi - wlo) >> fs) >= (uint64_t)TH_NFB) fs++;
            nfb = (int)((whi - wlo) >> fs) + 1;
            for (int i = threadIdx.x; i < nfb; i += TH_T) s_off[i] = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < rn; i += TH_T) {
                const uint64_t u = uoff(rrows[rbeg + i].key, P.lo);
                if (u >= wlo && u <= whi) atomicAdd(&s_off[(u - wlo) >> fs], 1u);
            }
            __syncthreads();
            uint32_t v[8];
            uint32_t sum = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int i = threadIdx.x * 8 + j;
                v[j] = i < nfb ? s_off[i] : 0u;
                sum += v[j];
            }
            uint32_t tot;
            uint32_t pre = block_excl_scan(sum, tmp32, &tot);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int i = threadIdx.x * 8 + j;
                if (i < nfb) s_off[i] = pre;
                pre += v[j];
            }
            __syncthreads();
            for (int i = threadIdx.x; i < rn; i += TH_T) {
                const Row<K, BAND> x = rrows[rbeg + i];
                const uint64_t u = uoff(x.key, P.lo);
                if (u >= wlo && u <= whi) {
                    const uint32_t pos = atomicAdd(&s_off[(u - wlo) >> fs], 1u);
                    s_ka[pos] = KA<K>{x.key, col_a<K, BAND>(x)};
                    s_p[pos] = x.pay;
                }
            }
            // bucket b now holds [b ? s_off[b-1] : 0, s_off[b])
        } else {
            for (int i = threadIdx.x; i < rn; i += TH_T) {
                const Row<K, BAND> x = rrows[rbeg + i];
                s_ka[i] = KA<K>{x.key, col_a<K, BAND>(x)};
                s_p[i] = x.pay;
            }
            if (threadIdx.x == 0) s_rows = (uint32_t)rn;
        }
        __syncthreads();

        unsigned long long acc = 0, csum = 0;
        const int rounds = (sn + TH_T - 1) / TH_T;
        // S rows stream through registers one round ahead: the next round's
        // row loads while this round's candidates are scanned
        Row<K, BAND> xn{};
        if ((int)threadIdx.x < sn) xn = srows[sbeg + threadIdx.x];
        for (int r = 0; r < rounds; r++) {
            const int j = r * TH_T + threadIdx.x;
            const Row<K, BAND> x = xn;
            if (j + TH_T < sn) xn = srows[sbeg + j + TH_T];
            uint32_t lo = 0, hi = 0;
            Interval<K> ia, ib;
            int32_t pay = 0;
            if (j < sn) {
                const K a = col_a<K, BAND>(x);
                pay = x.pay;
                ia = op_interval<K>(op, a);
                if (BAND) {
                    const K kk = x.key;
                    ib = band_interval<K>(kk, band);
                    const uint64_t u = uoff(kk, P.lo);
                    const uint64_t b = (uint64_t)band;
                    uint64_t ql = (u > b) ? u - b : 0;
                    uint64_t qh = (b > whi || u + b > whi || u + b < u) ? whi : u + b;
                    if (ql < wlo) ql = wlo;
                    const uint32_t b0 = (uint32_t)((ql - wlo) >> fs), b1 = (uint32_t)((qh - wlo) >> fs);
                    lo = b0 ? s_off[b0 - 1] : 0u;
                    hi = s_off[b1];
                } else {
                    lo = 0;
                    hi = s_rows;
                }
            }
            uint32_t m = 0;
            unsigned long long fs_sum = 0;
            if (MODE == MODE_EMIT) {
                // one scan: the matches among the first 32 candidates as a
                // mask, so the pairs are written without testing again; a
                // row with more candidates tests them again as it writes.
                // A warp without inverted intervals (!=, empty sets) takes
                // the bare range test.
                const bool plain = !__any_sync(0xffffffffu, j < sn && ia.inv);
                uint32_t mask = 0;
                m = plain ? theta_scan<true, false, K, BAND>(s_ka, s_p, lo, hi, ia, ib, &mask, &fs_sum)
                          : theta_scan<false, false, K, BAND>(s_ka, s_p, lo, hi, ia, ib, &mask, &fs_sum);
                const uint32_t incl = warp_incl_scan(m);
                const uint32_t wt = __shfl_sync(0xffffffffu, incl, 31);
                uint32_t base = 0;
                if (lane == 0 && wt) base = atomicAdd(&s_cursor, wt);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (m) {
                    jn_pair* o = out + item_off[it] + base + (incl - m);
                    if (hi - lo <= 32) {
                        while (mask) {
                            const int e = __ffs(mask) - 1;
                            mask &= mask - 1;
                            st_pair(o++, s_p[lo + e], pay);
                        }
                    } else if (plain) {
                        theta_emit_scan<true, K, BAND>(s_ka, s_p, lo, hi, ia, ib, o, pay);
                    } else {
                        theta_emit_scan<false, K, BAND>(s_ka, s_p, lo, hi, ia, ib, o, pay);
                    }
                }
            } else {
                const bool plain = !__any_sync(0xffffffffu, j < sn && ia.inv);
                uint32_t mask;
                m = plain ? theta_scan<true, MODE == MODE_AGG, K, BAND>(s_ka, s_p, lo, hi, ia, ib, &mask, &fs_sum)
                          : theta_scan<false, MODE == MODE_AGG, K, BAND>(s_ka, s_p, lo, hi, ia, ib, &mask, &fs_sum);
                acc += m;
                if (MODE == MODE_AGG && m) csum += fs_sum * chk_g(pay);
                if (record) {
                    // the row's pairs start where the warp's running cursor
                    // puts them; the emit pass writes them there
                    const uint32_t incl = warp_incl_scan(m);
                    const uint32_t wt = __shfl_sync(0xffffffffu, incl, 31);
                    uint32_t base = 0;
                    if (lane == 0 && wt) base = atomicAdd(&s_cursor, wt);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (j < sn) {
                        const bool narrow = hi - lo <= 32;
                        rec.rows[it * TH_SCH + j] =
                            make_uint2(mask, narrow ? ((base + incl - m) << 13) | lo : TH_WIDE);
                        if (!narrow) s_wide = 1;
                    }
                }
            }
        }
        if (record) {
            // a narrow item's offsets fit (at most TH_SCH * 32 pairs); its
            // staged payloads are what its records point into
            __syncthreads();
            const bool wide = s_wide != 0;
            if (!wide)
                for (int i = threadIdx.x; i < rn; i += TH_T) rec.pay[it * TH_RCAP + i] = s_p[i];
            if (threadIdx.x == 0) {
                rec.sdesc[it] = (sbeg << 14) | ((uint64_t)sn << 1) | (wide ? 1u : 0u);
                if (wide) atomicOr(rec.any_wide, 1u);
            }
        }
        if (MODE != MODE_EMIT) {
            const unsigned long long t = block_sum(acc, tmp64);
            if (MODE == MODE_AGG) {
                const unsigned long long cs = block_sum(csum, tmp64);
                if (threadIdx.x == 0 && cs) atomicAdd(chk, cs);
            }
            if (threadIdx.x == 0) item_val[it] = t;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------- cross regions --
// R rows whose group already decides "R.a op S.a" for S group y: up to two
// contiguous ranges of the partitioned R ([0, roff[y]) and [roff[y+1], nr)).
__device__ __forceinline__ void cross_ranges(int op, const uint64_t* roff, int y, int G, uint64_t* b0,
                                             uint64_t* l0, uint64_t* b1, uint64_t* l1) {
    const uint64_t below = roff[y], above_b = roff[y + 1], nr = roff[G];
    *b0 = 0; *l0 = 0; *b1 = above_b; *l1 = 0;
    switch (op) {
        case JN_LT: case JN_LE: *l0 = below; break;
        case JN_GT: case JN_GE: *l1 = nr - above_b; break;
        case JN_NE: case JN_ANY: *l0 = below; *l1 = nr - above_b; break;
        default: break;
    }
}

// cross[y] = pairs of y's cross regions; chunks[y] = ceil(cross[y] / CE_CHUNK).
__global__ void k_cross_counts(const uint64_t* __restrict__ roff, const uint64_t* __restrict__ soff,
                               int G, int op, uint64_t* __restrict__ cross, uint64_t* __restrict__ chunks) {
    int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= G) return;
    uint64_t b0, l0, b1, l1;
    cross_ranges(op, roff, y, G, &b0, &l0, &b1, &l1);
    const uint64_t c = (l0 + l1) * (soff[y + 1] - soff[y]);
    cross[y] = c;
    chunks[y] = (c + CE_CHUNK - 1) / CE_CHUNK;
}

// Checksum of the cross regions: sum_y (sum of f over the ranges) * (sum of g over S_y),
// using fpre = prefix sums of f over the partitioned R payloads.
template <typename R>
__global__ void k_cross_checksum(const uint64_t* __restrict__ roff, const uint64_t* __restrict__ soff,
                                 const R* __restrict__ srows, const uint64_t* __restrict__ fpre, int G,
                                 int op, unsigned long long* __restrict__ chk) {
    __shared__ unsigned long long tmp[33];
    const int y = blockIdx.x;
    uint64_t b0, l0, b1, l1;
    cross_ranges(op, roff, y, G, &b0, &l0, &b1, &l1);
    if (l0 + l1 == 0) return;
    unsigned long long g = 0;
    for (uint64_t i = soff[y] + threadIdx.x; i < soff[y + 1]; i += blockDim.x) g += chk_g(srows[i].pay);
    g = block_sum(g, tmp);
    if (threadIdx.x == 0) {
        const uint64_t f = (fpre[b0 + l0] - fpre[b0]) + (fpre[b1 + l1] - fpre[b1]);
        atomicAdd(chk, (unsigned long long)(f * g));
    }
}

template <typename R>
__global__ void k_fvals(const R* __restrict__ rows, int64_t n, uint64_t* __restrict__ f) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = chk_f(rows[i].pay);
}

// Writes the cross products: pair q of group y is (R[range(q % len)], S_y[q / len]).
template <typename R>
__global__ void __launch_bounds__(256)
k_cross_emit(const R* __restrict__ rrows, const uint64_t* __restrict__ roff, const R* __restrict__ srows,
             const uint64_t* __restrict__ soff, const uint64_t* __restrict__ cross_off,
             const uint64_t* __restrict__ chunk_prefix, int G, int op, uint64_t base,
             jn_pair* __restrict__ out, unsigned int* __restrict__ work) {
    __shared__ unsigned int s_item;
    const uint64_t nchunks = chunk_prefix[G];
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
        __syncthreads();
        const uint64_t it = s_item;
        __syncthreads();
        if (it >= nchunks) break;
        const int y = find_segment(chunk_prefix, G, it);
        uint64_t b0, l0, b1, l1;
        cross_ranges(op, roff, y, G, &b0, &l0, &b1, &l1);
        const uint64_t len = l0 + l1;
        const uint64_t total = len * (soff[y + 1] - soff[y]);
        const uint64_t q0 = (it - chunk_prefix[y]) * CE_CHUNK;
        const uint64_t q1 = min(total, q0 + CE_CHUNK);
        const uint64_t obase = base + cross_off[y];
        for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const uint64_t si = q / len, ri = q - si * len;
            const uint64_t r = ri < l0 ? b0 + ri : b1 + (ri - l0);
            st_pair(out + obase + q, rrows[r].pay, srows[soff[y] + si].pay);
        }
    }
}

template <typename K, bool HB>
static jn_status range_partition(jn_ctx* c, Scratch& s, const Cols<K>& T, const K* grp, const K* carry,
                                 const RangeParams* prm, int G, unsigned int* work, Row<K, HB>** orows,
                                 uint64_t** off) {
    const uint64_t n = (uint64_t)T.n;
    uint64_t *sb, *scn, *tp, *start;
    unsigned long long *hist, *cur;
    JN_TRY(s.get(&sb, 2));
    JN_TRY(s.get(&scn, 2));
    JN_TRY(s.get(&tp, 3));
    JN_TRY(s.get(&start, G + 1));
    JN_TRY(s.get(&hist, G));
    JN_TRY(s.get(&cur, G));
    JN_TRY(zero(c, hist, sizeof(unsigned long long) * G));
    JN_TRY(launch(c, K_SEGMENTS, k_one_segment, dim3(1), dim3(32), 0, sb, scn, tp, n));
    RangeDigit dg{prm};
    auto kh = k_seg_hist<K, RangeDigit>;
    const size_t smh = sizeof(uint32_t) * G;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kh, SC_T, smh);
    JN_TRY(launch(c, K_HIST, kh, dim3(max(per, 1) * c->num_sms), dim3(SC_T), smh, grp,
                  (const uint64_t*)sb, (const uint64_t*)scn, (const uint64_t*)tp, 1, dg, G, hist, work));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hist), start, G));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((G + 255) / 256), dim3(256), 0, (const uint64_t*)start,
                  cur, (int64_t)G));
    Row<K, HB>* rows;
    JN_TRY(s.get(&rows, n + 16));
    auto ks = k_scatter<K, HB, false, RangeDigit>;
    const size_t sm = scatter_smem<K, HB>();
    per = 0;
    ensure_smem((const void*)ks, sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ks, SC_T, sm);
    PartIn<K, HB> in{grp, carry, T.pay, nullptr, n, nullptr, nullptr};
    JN_TRY(launch(c, K_SCATTER, ks, dim3(max(per, 1) * c->num_sms), dim3(SC_T), sm, in, (const uint64_t*)sb,
                  (const uint64_t*)scn, (const uint64_t*)tp, 1, dg, G, (const uint32_t*)nullptr, 0u, cur, rows,
                  c->d_err));
    *orows = rows;
    *off = start;
    return JN_OK;
}

template <typename K, bool B>
static jn_status run_theta_t(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, int op, int64_t band, int mode,
                             OutPlan* plan, RunResult* res) {
    using RW = Row<K, B>;
    jn_run_info& info = c->info;
    int g = c->tune.theta_groups;
    if (g == 0) {
        const uint64_t base = B ? (uint64_t)R.n : (uint64_t)max(R.n, S.n);
        g = ceil_log2(ceil_div(base, B ? 1024 : 2048));
        if (g < 2) g = 2;
        if (g > 10) g = 10;
    }
    const int G = 1 << g;
    Scratch s(c);
    unsigned int* work;
    long long* mm;
    RangeParams* prm;
    uint64_t* d_small;
    JN_TRY(s.get(&work, 4));
    JN_TRY(s.get(&mm, 2));
    JN_TRY(s.get(&prm, 1));
    JN_TRY(s.get(&d_small, 4));
    JN_TRY(zero(c, d_small, 4 * sizeof(uint64_t)));
    const K* rg = B ? R.key2 : R.key;
    const K* sg = B ? S.key2 : S.key;
    JN_TRY(launch(c, K_MINMAX, k_mm_init, dim3(1), dim3(1), 0, mm));
    JN_TRY(launch(c, K_MINMAX, k_minmax<K>, dim3(2 * c->num_sms), dim3(512), 0, rg, R.n, mm));
    JN_TRY(launch(c, K_MINMAX, k_minmax<K>, dim3(2 * c->num_sms), dim3(512), 0, sg, S.n, mm));
    JN_TRY(launch(c, K_MINMAX, k_range_setup, dim3(1), dim3(1), 0, (const long long*)mm, G, prm));
    RW *rrows, *srows;
    uint64_t *roff, *soff;
    JN_TRY((range_partition<K, B>(c, s, R, rg, B ? R.key : nullptr, prm, G, work, &rrows, &roff)));
    JN_TRY((range_partition<K, B>(c, s, S, sg, B ? S.key : nullptr, prm, G, work, &srows, &soff)));
    // ---- compared regions (band window or diagonal) ----
    long long* d_band;
    int *d_op, *d_groups;
    JN_TRY(s.get(&d_band, 1));
    JN_TRY(s.get(&d_op, 2));
    d_groups = d_op + 1;
    JN_TRY(launch(c, K_MISC, k_set_theta_one, dim3(1), dim3(1), 0, d_band, d_op, d_groups,
                  (long long)(B ? band : -1), op, G));
    const ThetaSet ts{prm, d_band, d_op, d_groups, g};
    uint64_t *items, *ipre;
    JN_TRY(s.get(&items, G));
    JN_TRY(s.get(&ipre, G + 1));
    JN_TRY(launch(c, K_ITEMS, k_theta_items, dim3((G + 255) / 256), dim3(256), 0, (const uint64_t*)roff,
                  (const uint64_t*)soff, ts, G, items, (unsigned long long*)(d_small + 3)));
    JN_TRY(scan_u64(c, items, ipre, G));
    // ---- cross regions (one-column predicate only) ----
    uint64_t *cross = nullptr, *coff = nullptr, *chunks = nullptr, *cpre = nullptr;
    const bool has_cross = !B && op != JN_EQ;
    if (has_cross) {
        JN_TRY(s.get(&cross, G));
        JN_TRY(s.get(&coff, G + 1));
        JN_TRY(s.get(&chunks, G));
        JN_TRY(s.get(&cpre, G + 1));
        JN_TRY(launch(c, K_ITEMS, k_cross_counts, dim3((G + 255) / 256), dim3(256), 0,
                      (const uint64_t*)roff, (const uint64_t*)soff, G, op, cross, chunks));
        JN_TRY(scan_u64(c, cross, coff, G));
        JN_TRY(scan_u64(c, chunks, cpre, G));
    }
    JN_CUDA(c, cudaMemcpyAsync(d_small, ipre + G, 8, cudaMemcpyDeviceToDevice, c->stream));
    uint64_t h0[4];
    JN_TRY(read_back(c, d_small, h0, 4));
    const uint64_t nitems = h0[0], compared = h0[3];
    unsigned long long *ival, *chk;
    uint64_t* ioff;
    JN_TRY(s.get(&ival, nitems + 1));
    JN_TRY(s.get(&ioff, nitems + 1));
    JN_TRY(s.get(&chk, 1));
    JN_TRY(zero(c, chk, 8));
    const int cm = mode == MODE_AGG ? MODE_AGG : MODE_COUNT;
    auto pick = [&](int m) {
        if (m == MODE_EMIT) return k_theta_join<K, MODE_EMIT, B>;
        if (m == MODE_AGG) return k_theta_join<K, MODE_AGG, B>;
        return k_theta_join<K, MODE_COUNT, B>;
    };
    auto grid_of = [&](const void* fn, size_t smj) {
        int per = 0;
        ensure_smem(fn, smj);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, TH_T, smj);
        return max(per, 1) * c->num_sms;
    };
    // a band join that emits records every S row's matches in the count
    // pass (a few bytes per row and staged R row), so the emit pass gathers
    // them instead of staging and testing again
    ThetaRec rec{nullptr, nullptr, nullptr, nullptr};
    if (B && mode == MODE_EMIT && nitems && nitems <= (uint64_t)(4ull << 30) / (TH_SCH * 8 + TH_RCAP * 4)) {
        JN_TRY(s.get(&rec.rows, nitems * TH_SCH));
        JN_TRY(s.get(&rec.pay, nitems * TH_RCAP));
        JN_TRY(s.get(&rec.sdesc, nitems));
        rec.any_wide = reinterpret_cast<unsigned int*>(d_small + 2);
        JN_TRY(zero(c, d_small + 2, 8));
        // the gather reads the saved payloads as 16-byte words
        if ((uintptr_t)rec.pay & 15) rec = ThetaRec{nullptr, nullptr, nullptr, nullptr};
    }
    if (nitems) {
        auto kc = pick(cm);
        JN_TRY(zero(c, work, 4));
        JN_TRY(launch(c, K_THETA_COUNT, kc, dim3(grid_of((const void*)kc, theta_smem<K>(cm))), dim3(TH_T),
                      theta_smem<K>(cm), (const RW*)rrows,
                      (const uint64_t*)roff, (const RW*)srows, (const uint64_t*)soff, ts, G, (const uint64_t*)ipre,
                      ival, chk, (const uint64_t*)nullptr, (jn_pair*)nullptr, work, rec));
    }
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(ival), ioff, (int64_t)nitems));
    if (has_cross && mode == MODE_AGG) {
        uint64_t *fv, *fpre;
        JN_TRY(s.get(&fv, R.n));
        JN_TRY(s.get(&fpre, R.n + 1));
        JN_TRY(launch(c, K_MISC, k_fvals<RW>, dim3((unsigned)ceil_div(R.n, 256)), dim3(256), 0, (const RW*)rrows,
                      (int64_t)R.n, fv));
        JN_TRY(scan_u64(c, fv, fpre, R.n));
        JN_TRY(launch(c, K_MISC, k_cross_checksum<RW>, dim3(G), dim3(256), 0, (const uint64_t*)roff,
                      (const uint64_t*)soff, (const RW*)srows, (const uint64_t*)fpre, G, op, chk));
    }
    JN_CUDA(c, cudaMemcpyAsync(d_small, ioff + nitems, 8, cudaMemcpyDeviceToDevice, c->stream));
    JN_CUDA(c, cudaMemcpyAsync(d_small + 1, chk, 8, cudaMemcpyDeviceToDevice, c->stream));
    if (has_cross) JN_CUDA(c, cudaMemcpyAsync(d_small + 2, coff + G, 8, cudaMemcpyDeviceToDevice, c->stream));
    uint64_t h[3] = {0, 0, 0};
    JN_TRY(read_back(c, d_small, h, (has_cross || rec.rows) ? 3 : 2));
    const bool any_wide = rec.rows && (h[2] & 0xffffffffu) != 0;
    const uint64_t diag = h[0], crossn = has_cross ? h[2] : 0;
    const uint64_t total = diag + crossn;
    res->count = total;
    res->checksum = h[1];
    info.result = total;
    info.partitions = (uint64_t)G;
    info.work_items = nitems;
    info.r_survivors = (uint64_t)R.n;
    info.s_survivors = (uint64_t)S.n;
    info.prefilter = 0;
    info.cartesian_bound = compared + crossn;  // cross regions are written whole
    if (mode != MODE_EMIT) return JN_OK;
    JN_TRY(out_prepare(c, s, total, *plan));
    if constexpr (B) {
        if (diag && rec.rows)
            JN_TRY(launch(c, K_THETA_GATHER, k_theta_gather<K>,
                          dim3((unsigned)min(nitems, (uint64_t)8 * c->num_sms)), dim3(TH_T), 0, (const RW*)srows,
                          (const uint64_t*)(ipre + G), (const uint64_t*)ioff, rec, plan->dev));
    }
    if (diag && (!rec.rows || any_wide)) {
        // every item, or (after the gather) the wide ones
        auto ke = pick(MODE_EMIT);
        JN_TRY(zero(c, work, 4));
        JN_TRY(launch(c, K_THETA_EMIT, ke, dim3(grid_of((const void*)ke, theta_smem<K>(MODE_EMIT))), dim3(TH_T),
                      theta_smem<K>(MODE_EMIT), (const RW*)rrows,
                      (const uint64_t*)roff, (const RW*)srows, (const uint64_t*)soff, ts, G, (const uint64_t*)ipre,
                      (unsigned long long*)nullptr, (unsigned long long*)nullptr, (const uint64_t*)ioff, plan->dev,
                      work, rec));
    }
    if (crossn) {
        JN_TRY(zero(c, work, 4));
        JN_TRY(launch(c, K_CROSS_EMIT, k_cross_emit<RW>, dim3(4 * c->num_sms), dim3(256), 0, (const RW*)rrows,
                      (const uint64_t*)roff, (const RW*)srows, (const uint64_t*)soff, (const uint64_t*)coff,
                      (const uint64_t*)cpre, G, op, diag, plan->dev, work));
    }
    JN_TRY(out_finish(c, total, *plan));
    return JN_OK;
}

template <typename K>
jn_status run_theta(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, int op, int64_t band, int mode,
                    OutPlan* plan, RunResult* res) {
    if (R.n == 0 || S.n == 0) {
        res->count = res->checksum = 0;
        if (mode == MODE_EMIT) {
            Scratch s0(c);
            JN_TRY(out_prepare(c, s0, 0, *plan));
            JN_TRY(out_finish(c, 0, *plan));
        }
        return JN_OK;
    }
    if (band >= 0) return run_theta_t<K, true>(c, R, S, op, band, mode, plan, res);
    return run_theta_t<K, false>(c, R, S, op, band, mode, plan, res);
}

// ------------------------------------------------------------- batches --
// Digit of a batch's range pass: segment s belongs to join s % m, whose
// range parameters give the group.
struct SegRangeDigit {
    static constexpr int kFilterWords = 0;
    const RangeParams* prm;
    int m;
    long long lo;
    int shift;
    __device__ __forceinline__ void bind(uint32_t*) {}
    __device__ __forceinline__ void set_seg(int s) {
        const RangeParams& p = prm[s % m];
        lo = p.lo;
        shift = p.shift;
    }
    __device__ __forceinline__ bool is_special(uint32_t) const { return false; }
    template <typename K>
    __device__ __forceinline__ uint32_t operator()(K k) const {
        return (uint32_t)(((uint64_t)((int64_t)k - lo)) >> shift);
    }
};

__global__ void k_bmm_init(long long* mm, int m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        mm[2 * i] = LLONG_MAX;
        mm[2 * i + 1] = LLONG_MIN;
    }
}

// Per-join minimum and maximum of the grouped column over both tables.
template <typename K>
__global__ void k_batch_minmax(const SegCols<K>* __restrict__ segs, const TileRef* __restrict__ tiles,
                               const uint64_t* __restrict__ ntiles_p, int m, long long* __restrict__ mm) {
    const uint64_t ntiles = *ntiles_p;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileRef x = tiles[t];
        const K* k = segs[x.seg].key;
        long long lo = LLONG_MAX, hi = LLONG_MIN;
        for (int i = threadIdx.x; i < x.cnt; i += blockDim.x) {
            const long long v = (long long)k[x.beg + i];
            lo = v < lo ? v : lo;
            hi = v > hi ? v : hi;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long a = __shfl_xor_sync(0xffffffffu, lo, o);
            const long long b = __shfl_xor_sync(0xffffffffu, hi, o);
            lo = a < lo ? a : lo;
            hi = b > hi ? b : hi;
        }
        if ((threadIdx.x & 31) == 0 && lo <= hi) {
            atomicMin(&mm[2 * (x.seg % m)], lo);
            atomicMax(&mm[2 * (x.seg % m) + 1], hi);
        }
    }
}

__global__ void k_batch_range_setup(const long long* __restrict__ mm, const int* __restrict__ groups, int m,
                                    RangeParams* __restrict__ p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    long long lo = mm[2 * i], hi = mm[2 * i + 1];
    if (lo > hi) { lo = 0; hi = 0; }
    const uint64_t span = (uint64_t)hi - (uint64_t)lo;
    int s = 0;
    while (s < 63 && (span >> s) >= (uint64_t)groups[i]) s++;
    p[i].lo = lo;
    p[i].hi = hi;
    p[i].shift = s;
    p[i].groups = (int)(span >> s) + 1;
    p[i].fshift = 0;
    p[i].pad = 0;
}

template <typename K, typename Digit>
__global__ void __launch_bounds__(SC_T)
k_batch_hist_any(const SegCols<K>* __restrict__ segs, const TileRef* __restrict__ tiles,
                 const uint64_t* __restrict__ ntiles_p, Digit dg, unsigned long long* __restrict__ hist) {
    __shared__ uint32_t s_h[SC_FMAX];
    const uint64_t ntiles = *ntiles_p;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileRef x = tiles[t];
        dg.set_seg(x.seg);
        for (int i = threadIdx.x; i < SC_FMAX; i += blockDim.x) s_h[i] = 0;
        __syncthreads();
        const K* k = segs[x.seg].key;
        for (int i = threadIdx.x; i < x.cnt; i += blockDim.x) atomicAdd(&s_h[dg(k[x.beg + i])], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < SC_FMAX; i += blockDim.x)
            if (s_h[i]) atomicAdd(&hist[(uint64_t)x.seg * SC_FMAX + i], (unsigned long long)s_h[i]);
        __syncthreads();
    }
}

__global__ void k_band_offsets(const uint64_t* __restrict__ item_prefix, const uint64_t* __restrict__ ioff,
                               int count, uint64_t* __restrict__ out_off) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > count) return;
    out_off[i] = ioff[item_prefix[(uint64_t)i * SC_FMAX]];
}

__global__ void k_set_words(long long* band, int* op, int* groups, const long long* hb, const int* hop,
                            const int* hg, int m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        band[i] = hb[i];
        op[i] = hop[i];
        groups[i] = hg[i];
    }
}

// A batch of band joins run as one: join i's R table is segment i and its S
// table segment m + i of one range pass on column k, join i owns partitions
// [i * 1024, i * 1024 + groups_i), and the count and emit passes run over one
// work queue of (join, group, R chunk, S chunk) items of all joins.
template <typename K>
struct BandBatchRun : BatchRun {
    using RW = Row<K, true>;
    std::unique_ptr<Scratch> s;
    int m = 0;
    uint64_t P = 0, nitems = 0;
    RW* prow = nullptr;
    uint64_t *start = nullptr, *ipre = nullptr, *ioff = nullptr;
    ThetaSet ts{};
    unsigned int* work = nullptr;
    size_t smj = 0;

    jn_status prepare(jn_ctx* c, const Cols<K>* Rs, const Cols<K>* Ss, const int* ops, const int64_t* bands) {
        s.reset(new Scratch(c));
        std::vector<SegCols<K>> segs(2 * (size_t)m);
        std::vector<TileRef> tiles;
        std::vector<int> groups(m), hop(m);
        std::vector<long long> hb(m);
        uint64_t rows = 0;
        for (int i = 0; i < m; i++) {
            int g = ceil_log2(ceil_div((uint64_t)max(Rs[i].n, (int64_t)1), 1024));
            if (g < 2) g = 2;
            if (g > 10) g = 10;
            groups[i] = 1 << g;
            hop[i] = ops[i];
            hb[i] = bands[i];
            segs[i] = SegCols<K>{Rs[i].key2, Rs[i].key, Rs[i].pay, (uint64_t)Rs[i].n};
            segs[m + i] = SegCols<K>{Ss[i].key2, Ss[i].key, Ss[i].pay, (uint64_t)Ss[i].n};
            rows += (uint64_t)Rs[i].n + (uint64_t)Ss[i].n;
        }
        for (int sgi = 0; sgi < 2 * m; sgi++)
            for (uint64_t b = 0; b < segs[sgi].n; b += SC_TILE)
                tiles.push_back(TileRef{b, sgi, (int)min((uint64_t)SC_TILE, segs[sgi].n - b)});
        const uint64_t ntiles = tiles.size();
        P = (uint64_t)m * SC_FMAX;
        SegCols<K>* d_segs;
        TileRef* d_tiles;
        uint64_t *d_ntiles, *items;
        long long *mm, *d_band, *h_band;
        int *d_op, *d_groups, *h_op, *h_groups;
        RangeParams* prm;
        unsigned long long *hist, *cur;
        JN_TRY(s->get(&d_segs, 2 * (size_t)m));
        JN_TRY(s->get(&d_tiles, ntiles + 1));
        JN_TRY(s->get(&d_ntiles, 1));
        JN_TRY(s->get(&mm, 2 * (size_t)m));
        JN_TRY(s->get(&prm, (size_t)m));
        JN_TRY(s->get(&d_band, (size_t)m));
        JN_TRY(s->get(&h_band, (size_t)m));
        JN_TRY(s->get(&d_op, (size_t)m));
        JN_TRY(s->get(&h_op, (size_t)m));
        JN_TRY(s->get(&d_groups, (size_t)m));
        JN_TRY(s->get(&h_groups, (size_t)m));
        JN_TRY(s->get(&hist, 2 * P));
        JN_TRY(s->get(&start, 2 * P + 1));
        JN_TRY(s->get(&cur, 2 * P));
        JN_TRY(s->get(&prow, rows + 16));
        JN_TRY(s->get(&items, P));
        JN_TRY(s->get(&ipre, P + 1));
        JN_TRY(s->get(&work, 4));
        JN_CUDA(c, cudaMemcpyAsync(d_segs, segs.data(), sizeof(SegCols<K>) * segs.size(), cudaMemcpyHostToDevice,
                                   c->stream));
        if (ntiles)
            JN_CUDA(c, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TileRef) * ntiles, cudaMemcpyHostToDevice,
                                       c->stream));
        JN_CUDA(c, cudaMemcpyAsync(d_ntiles, &ntiles, sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream));
        JN_CUDA(c, cudaMemcpyAsync(h_band, hb.data(), sizeof(long long) * m, cudaMemcpyHostToDevice, c->stream));
        JN_CUDA(c, cudaMemcpyAsync(h_op, hop.data(), sizeof(int) * m, cudaMemcpyHostToDevice, c->stream));
        JN_CUDA(c, cudaMemcpyAsync(h_groups, groups.data(), sizeof(int) * m, cudaMemcpyHostToDevice, c->stream));
        JN_CUDA(c, cudaStreamSynchronize(c->stream));  // the host vectors go out of scope below
        ts = ThetaSet{prm, d_band, d_op, d_groups, 10};
        smj = theta_smem<K>(MODE_COUNT);

        // ---- phase 1a: ranges, range partition and work items ----
        {
            GraphPhase gp(c, c->tune.graphs != 0 && !c->profiling);
            JN_TRY(gp.begin());
            jn_status st = JN_OK;
            do {
                const unsigned gm = (unsigned)ceil_div((uint64_t)m, 256);
                if ((st = launch(c, K_MISC, k_set_words, dim3(gm), dim3(256), 0, d_band, d_op, d_groups,
                                 (const long long*)h_band, (const int*)h_op, (const int*)h_groups, m)) != JN_OK)
                    break;
                if ((st = launch(c, K_MINMAX, k_bmm_init, dim3(gm), dim3(256), 0, mm, m)) != JN_OK) break;
                if ((st = launch(c, K_MINMAX, k_batch_minmax<K>, dim3(4 * c->num_sms), dim3(256), 0,
                                 (const SegCols<K>*)d_segs, (const TileRef*)d_tiles, (const uint64_t*)d_ntiles, m,
                                 mm)) != JN_OK)
                    break;
                if ((st = launch(c, K_MINMAX, k_batch_range_setup, dim3(gm), dim3(256), 0, (const long long*)mm,
                                 (const int*)d_groups, m, prm)) != JN_OK)
                    break;
                SegRangeDigit dg{prm, m, 0, 0};
                if ((st = zero(c, hist, sizeof(unsigned long long) * 2 * P)) != JN_OK) break;
                if ((st = launch(c, K_HIST, k_batch_hist_any<K, SegRangeDigit>, dim3(4 * c->num_sms), dim3(SC_T), 0,
                                 (const SegCols<K>*)d_segs, (const TileRef*)d_tiles, (const uint64_t*)d_ntiles, dg,
                                 hist)) != JN_OK)
                    break;
                if ((st = scan_u64(c, reinterpret_cast<const uint64_t*>(hist), start, (int64_t)(2 * P))) != JN_OK)
                    break;
                if ((st = launch(c, K_MISC, k_init_cursor, dim3((unsigned)ceil_div(2 * P, 256)), dim3(256), 0,
                                 (const uint64_t*)start, cur, (int64_t)(2 * P))) != JN_OK)
                    break;
                auto ks = k_scatter<K, true, false, SegRangeDigit>;
                const size_t sm = scatter_smem<K, true>();
                ensure_smem((const void*)ks, sm);
                int per = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ks, SC_T, sm);
                PartIn<K, true> in{nullptr, nullptr, nullptr, nullptr, 0, d_segs, d_tiles};
                if ((st = launch(c, K_SCATTER, ks, dim3(max(per, 1) * c->num_sms), dim3(SC_T), sm, in,
                                 (const uint64_t*)nullptr, (const uint64_t*)nullptr, (const uint64_t*)d_ntiles, 0, dg,
                                 SC_FMAX, (const uint32_t*)nullptr, 0u, cur, prow, c->d_err)) != JN_OK)
                    break;
                if ((st = launch(c, K_ITEMS, k_theta_items, dim3((unsigned)ceil_div(P, 256)), dim3(256), 0,
                                 (const uint64_t*)start, (const uint64_t*)(start + P), ts, (int)P, items,
                                 (unsigned long long*)nullptr)) != JN_OK)
                    break;
                if ((st = scan_u64(c, items, ipre, (int64_t)P)) != JN_OK) break;
            } while (0);
            if (st != JN_OK) {
                gp.abort();
                return st;
            }
            JN_TRY(gp.end_and_run());
        }
        uint64_t* d_small;
        JN_TRY(s->get(&d_small, 2));
        JN_CUDA(c, cudaMemcpyAsync(d_small, ipre + P, 8, cudaMemcpyDeviceToDevice, c->stream));
        JN_TRY(read_back(c, d_small, &nitems, 1));
        // ---- phase 1b: count pass, scan, per-join offsets ----
        unsigned long long *ival, *chk;
        uint64_t* d_off;
        JN_TRY(s->get(&ival, nitems + 1));
        JN_TRY(s->get(&ioff, nitems + 1));
        JN_TRY(s->get(&chk, 1));
        JN_TRY(s->get(&d_off, (size_t)m + 1));
        {
            GraphPhase gp(c, c->tune.graphs != 0 && !c->profiling);
            JN_TRY(gp.begin());
            jn_status st = JN_OK;
            do {
                if ((st = zero(c, chk, 8)) != JN_OK) break;
                if ((st = zero(c, work, 4)) != JN_OK) break;
                if (nitems) {
                    auto kc = k_theta_join<K, MODE_COUNT, true>;
                    ensure_smem((const void*)kc, smj);
                    int per = 0;
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kc, TH_T, smj);
                    if ((st = launch(c, K_THETA_COUNT, kc, dim3(max(per, 1) * c->num_sms), dim3(TH_T), smj,
                                     (const RW*)prow, (const uint64_t*)start, (const RW*)prow,
                                     (const uint64_t*)(start + P), ts, (int)P, (const uint64_t*)ipre, ival, chk,
                                     (const uint64_t*)nullptr, (jn_pair*)nullptr, work,
                                     ThetaRec{nullptr, nullptr, nullptr, nullptr})) != JN_OK)
                        break;
                }
                if ((st = scan_u64(c, reinterpret_cast<const uint64_t*>(ival), ioff, (int64_t)nitems)) != JN_OK) break;
                if ((st = launch(c, K_MISC, k_band_offsets, dim3((unsigned)ceil_div((uint64_t)m + 1, 256)), dim3(256),
                                 0, (const uint64_t*)ipre, (const uint64_t*)ioff, m, d_off)) != JN_OK)
                    break;
            } while (0);
            if (st != JN_OK) {
                gp.abort();
                return st;
            }
            JN_TRY(gp.end_and_run());
        }
        offsets.assign((size_t)m + 1, 0);
        JN_CUDA(c, cudaMemcpyAsync(offsets.data(), d_off, sizeof(uint64_t) * (m + 1), cudaMemcpyDeviceToHost,
                                   c->stream));
        uint64_t dummy;
        JN_TRY(read_back(c, d_small, &dummy, 0));
        total = offsets[m];
        return JN_OK;
    }

    jn_status emit(jn_ctx* c, jn_pair* out) override {
        if (total == 0) return JN_OK;
        GraphPhase gp(c, c->tune.graphs != 0 && !c->profiling);
        JN_TRY(gp.begin());
        jn_status st = zero(c, work, 4);
        if (st == JN_OK) {
            auto ke = k_theta_join<K, MODE_EMIT, true>;
            const size_t sme = theta_smem<K>(MODE_EMIT);
            ensure_smem((const void*)ke, sme);
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ke, TH_T, sme);
            st = launch(c, K_THETA_EMIT, ke, dim3(max(per, 1) * c->num_sms), dim3(TH_T), sme, (const RW*)prow,
                        (const uint64_t*)start, (const RW*)prow, (const uint64_t*)(start + P), ts, (int)P,
                        (const uint64_t*)ipre, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                        (const uint64_t*)ioff, out, work, ThetaRec{nullptr, nullptr, nullptr, nullptr});
        }
        if (st != JN_OK) {
            gp.abort();
            return st;
        }
        JN_TRY(gp.end_and_run());
        return JN_OK;
    }
};

template <typename K>
jn_status batch_band_prepare(jn_ctx* c, int m, const Cols<K>* Rs, const Cols<K>* Ss, const int* ops,
                             const int64_t* bands, std::unique_ptr<BatchRun>* run) {
    std::unique_ptr<BandBatchRun<K>> r(new BandBatchRun<K>());
    r->m = m;
    JN_TRY(r->prepare(c, Rs, Ss, ops, bands));
    c->info.partitions += r->P;
    c->info.work_items += r->nitems;
    run->reset(r.release());
    return JN_OK;
}

template jn_status batch_band_prepare<int32_t>(jn_ctx*, int, const Cols<int32_t>*, const Cols<int32_t>*, const int*,
                                               const int64_t*, std::unique_ptr<BatchRun>*);
template jn_status batch_band_prepare<int64_t>(jn_ctx*, int, const Cols<int64_t>*, const Cols<int64_t>*, const int*,
                                               const int64_t*, std::unique_ptr<BatchRun>*);

template jn_status run_theta<int32_t>(jn_ctx*, const Cols<int32_t>&, const Cols<int32_t>&, int, int64_t,
                                      int, OutPlan*, RunResult*);
template jn_status run_theta<int64_t>(jn_ctx*, const Cols<int64_t>&, const Cols<int64_t>&, int, int64_t,
                                      int, OutPlan*, RunResult*);

}  // namespace jnx
