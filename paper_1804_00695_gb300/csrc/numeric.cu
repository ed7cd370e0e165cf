// Numeric phase (Section 2.1): C_i = sum over stored a_ik of a_ik * B_k.
// Rows are binned by their exact output count (known from the symbolic
// phase) and their products:
//
// * bins 1-2 (<= 32 outputs): groups of G lanes per row, a shared-memory
//   hash map from column to value per row (the sparse hash accumulators of
//   Section 2.1), products dealt evenly over the lanes;
// * bins 3-4 (<= 1024 outputs): a warp per row with a dense rank
//   accumulator over the row's column span (bitmap, prefix counts, values
//   by rank) when the span is at most 2048 blocks of 32 columns (three
//   bitmap sizes), else a warp-level shared hash map;
// * bin 5 (<= 4096 outputs): a block per row, shared hash map;
// * bin 6 (more): a windowed dense accumulator when the rows of B are
//   sorted, else a two-level hash map (shared, then global memory: Section
//   3.3's multilevel memory).
//
// Output rows have ascending columns.  FP64 values are accumulated as
// double-words (two floats, 48 significand bits: dword.cuh) in the FP32
// pipeline unless an input lies outside the double-word range, in which
// case that row (or, for B, the whole call) uses native FP64; the block
// kernels accumulate in native precision.
#include <climits>
#include <type_traits>
#include "dword.cuh"
#include "internal.cuh"

namespace sg {

enum { MODE_F32 = 0, MODE_DW = 1, MODE_F64 = 2 };

struct NumP {
    const int64_t *arp; const int32_t *acol; const void *aval;
    const int64_t *brp; const int32_t *bcol; const void *bval; const float2 *bsplit;
    const int64_t *crp; int32_t *ccol; void *cval;
};

// Find or insert `col` in a map of 2^L slots (keys only); -1 if full.
__device__ __forceinline__ int map_slot(int *keys, int L, int col) {
    const unsigned msk = (1u << L) - 1;
    unsigned h = hash_slot(col, L);
#pragma unroll 1
    for (int probe = 0; probe <= (int)msk; probe++) {
        int k = ((volatile int *)keys)[h];
        if (k == col) return (int)h;
        if (k == -1) {
            int old = atomicCAS(&keys[h], -1, col);
            if (old == -1 || old == col) return (int)h;
        }
        h = (h + 1) & msk;
    }
    return -1;
}

__device__ __forceinline__ int next_pow2(int n) { return n <= 1 ? 1 : 1 << (32 - __clz(n - 1)); }

// B values split once into double-words; flags the call if any value is
// outside the double-word range.
__global__ void k_split_values(int64_t nnz, const double *__restrict__ v, float2 *__restrict__ out,
                               DevState *st) {
    bool ok = true;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dw_split(v[i], ok);
    if (!ok) atomicOr(&st->b_out_of_range, 1);
}

// Accumulator slot: 4 bytes (FP32) or 8 bytes (a double or a double-word).
template <int MODE>
using SlotT = typename std::conditional<MODE == MODE_F32, float, double>::type;

// Value type of A and B elements.
template <int MODE>
using ValT = typename std::conditional<MODE == MODE_F32, float, double>::type;

template <int MODE>
__device__ __forceinline__ void acc_update(SlotT<MODE> *acc, int slot, bool nat, const void *bval,
                                           const float2 *bsplit, int64_t q, ValT<MODE> av, float2 a2) {
    if (MODE == MODE_F32) {
        acc[slot] += av * ((const float *)bval)[q];
    } else if (MODE == MODE_DW && !nat) {
        float2 *a = (float2 *)acc;
        a[slot] = dw_add(a[slot], dw_mul(a2, bsplit[q]));
    } else {
        acc[slot] += av * ((const double *)bval)[q];
    }
}

template <int MODE>
__device__ __forceinline__ void store_out(void *cval, int64_t pos, SlotT<MODE> v, bool nat) {
    if (MODE == MODE_F32) {
        ((float *)cval)[pos] = v;
    } else if (MODE == MODE_DW && !nat) {
        // the slot holds a double-word: hi in the low 32 bits, lo in the high 32
        const unsigned long long bits = (unsigned long long)__double_as_longlong((double)v);
        ((double *)cval)[pos] = dw_to_double(__uint_as_float((unsigned)bits),
                                             __uint_as_float((unsigned)(bits >> 32)));
    } else {
        ((double *)cval)[pos] = v;
    }
}

template <int MODE>
__device__ __forceinline__ ValT<MODE> load_a(const void *aval, int64_t p) {
    return ((const ValT<MODE> *)aval)[p];
}

// Three-level accumulation of a double-word product p into a slot held by
// one thread: the high float takes p.x and its exact rounding error (TwoSum)
// joins p.y; that sum goes to the second float the same way; the last, tiny
// residue is added to a third float.  Every rounding of the first two levels
// is recovered exactly, so an entry with n terms ends within
// (6 + n^3 2^-24) 2^-48 sum|a_ik||b_kj| of the exact sum, product errors
// included, in any order of the updates.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void acc3_add(float &hi, float &lo, float &lo2, float2 p) {
    float s1, e1, t, f, s2, e2;
    two_sum(hi, p.x, s1, e1);
    two_sum(e1, p.y, t, f);
    two_sum(lo, t, s2, e2);
    hi = s1;
    lo = s2;
    lo2 = __fadd_rn(lo2, __fadd_rn(e2, f));
}

// The same three levels updated by atomic adds, for slots shared by lanes
// that may add to them at once: the returned old values give the exact
// rounding errors of the first two levels.
__device__ __forceinline__ void dw_atomic_acc(float2 *v2, float *v3, int slot, float2 p) {
    float s1, e1, t, f, s2, e2;
    const float o1 = atomicAdd(&v2[slot].x, p.x);
    two_sum(o1, p.x, s1, e1);
    two_sum(e1, p.y, t, f);
    const float o2 = atomicAdd(&v2[slot].y, t);
    two_sum(o2, t, s2, e2);
    atomicAdd(&v3[slot], __fadd_rn(e2, f));
}

// vals[slot] += v for every lane with `valid`, where vals is private to the
// warp.  Lanes that hit the same slot first sum their values in lane order
// (one __match_any_sync, then as many shuffles as the largest group has
// members), so that one lane per slot writes and the write is a plain
// load-add-store: no atomic, and no retries when several products of one
// step meet in one slot.  Called by all 32 lanes.
__device__ __forceinline__ void warp_acc_f64(double *vals, int slot, bool valid, double v, int lane) {
    const unsigned grp = __match_any_sync(0xffffffffu, valid ? slot : -1 - lane);
    const int leader = __ffs(grp) - 1;
    const int m = __popc(grp);
    const int maxm = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
    unsigned rest = grp & (grp - 1);   // members after the leader
    double sum = v;
    for (int k = 1; k < maxm; k++) {
        const int src = rest ? __ffs(rest) - 1 : lane;
        rest &= rest - 1;
        const double x = __shfl_sync(0xffffffffu, v, src);
        if (k < m) sum += x;
    }
    if (valid && lane == leader) vals[slot] += sum;
    __syncwarp();
}

// Final value of a three-level slot as a double.
__device__ __forceinline__ double dw3_to_double(float hi, float lo, float lo2) {
    float s, e;
    two_sum(hi, __fadd_rn(lo, lo2), s, e);
    return dw_to_double(s, e);
}

// Adds one product to a slot held by this thread.  FP32: px.  Double-word:
// (px, py); rows with at most DW2_MAX_TERMS stored a_ik (so at most that many
// terms per entry) use the two-float accumulate dw_add, whose error stays
// within (7 + 5n) 2^-48 sum|a||b| <= 1e-12 sum|a||b|; longer rows use the
// three-level acc3_add.  Native FP64: (px, py) are the low and high words of
// the product, and the slot keeps a double's words in hi and lo.
constexpr int DW2_MAX_TERMS = 48;

template <int MODE>
__device__ __forceinline__ void acc_slot(float *hi, float *lo, float *lo2, int slot, bool nat,
                                         bool three, float px, float py) {
    if (MODE == MODE_F32) {
        hi[slot] += px;
    } else if (MODE == MODE_DW && !nat) {
        if (three) {
            acc3_add(hi[slot], lo[slot], lo2[slot], make_float2(px, py));
        } else {
            const float2 r = dw_add(make_float2(hi[slot], lo[slot]), make_float2(px, py));
            hi[slot] = r.x;
            lo[slot] = r.y;
        }
    } else {
        const double v = __hiloint2double(__float_as_int(lo[slot]), __float_as_int(hi[slot])) +
                         __hiloint2double(__float_as_int(py), __float_as_int(px));
        hi[slot] = __int_as_float(__double2loint(v));
        lo[slot] = __int_as_float(__double2hiint(v));
    }
}

// Bins 1-2: a warp takes 32/G consecutive rows, G lanes per row, map of up
// to 64 slots per row.  The products of a row are dealt out evenly: the
// stored a_ik are staged E at a time in shared memory with the prefix sums
// of nnz(B_k), and in each step the G lanes take G consecutive products
// (lane l the t-th, t = step*G + l), finding their a_ik with a cursor that
// only moves forward.  Loads of B stay coalesced within each B_k.  Products
// are added to their slot with shared-memory atomics; double-words keep
// three levels whose rounding errors are recovered exactly from the old
// values the atomics return.  The occupied slots are then compacted and
// each row written in ascending column order (rank by counting).
// Per-row-slot layout of k_num_small in 32-bit words: hi[SMAX], lo[SMAX],
// lo2[SMAX], keys[SMAX], eq0[E] (int64), ea[E] (double), pre[E+1].  The
// stride is padded to G (mod 32) words so that the 32/G row slots of a warp
// start on different banks.
template <int G>
struct SmallLayout {
    static constexpr int SMAX = 64, E = 32;
    static constexpr int raw = 4 * SMAX + 2 * E + 2 * E + E + 1;
    static constexpr int stride = G == 32 ? ((raw + 1) & ~1) : raw + ((G - raw % 32) + 32) % 32;
    static_assert(stride % 2 == 0, "8-byte arrays need an even stride");
};

template <int G, int MODE>
__global__ void __launch_bounds__(256, G <= 4 ? 2 : 4) k_num_small(NumP a, const int4 *__restrict__ bdesc, int64_t n,
                                                   const uint8_t *__restrict__ bins,
                                                   const DevState *st, int *err, int maxbin,
                                                   int slot_factor) {
    constexpr int SMAX = SmallLayout<G>::SMAX, RPW = 32 / G, WPB = 8, PER = SMAX / G;
    constexpr int E = SmallLayout<G>::E, EL = E / G;   // entries staged per batch, per lane
    using V = ValT<MODE>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / G, gl = lane % G, gbase = g * G;
    const int rs = w * RPW + g;   // row slot in the block
    int *reg = (int *)smem_raw + rs * SmallLayout<G>::stride;
    float *hi = (float *)reg;
    float *lo = hi + SMAX;
    float *lo2 = lo + SMAX;
    double *dv = (double *)reg;   // native FP64 slots (hi and lo together)
    int *keys = (int *)(lo2 + SMAX);
    long long *eq0 = (long long *)(keys + SMAX);
    double *ea = (double *)(eq0 + E);
    int *pre = (int *)(ea + E);
    // native FP64 rows keep a double's low word in hi[] and its high word in lo[]
    const unsigned lmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1);
    const bool b_bad = MODE == MODE_DW && st->b_out_of_range;
    int flag = 0;
    const int64_t stride = (int64_t)gridDim.x * WPB * RPW;
    for (int64_t base = ((int64_t)blockIdx.x * WPB + w) * RPW; base < n; base += stride) {
        const int64_t i = base + g;
        const int bi = i < n ? bins[i] : 0;
        const bool active = bi >= 1 && bi <= maxbin;
        const int64_t p0 = active ? a.arp[i] : 0;
        const int plen = active ? (int)(a.arp[i + 1] - p0) : 0;
        const int64_t out = active ? a.crp[i] : 0;
        const int nn = active ? (int)(a.crp[i + 1] - out) : 0;
        int S = next_pow2(slot_factor * nn);
        S = S < 8 ? 8 : (S > SMAX ? SMAX : S);
        const int L = __ffs(S) - 1;
#pragma unroll
        for (int t = 0; t < PER; t++) {
            const int sidx = gl + t * G;
            if (t * G >= S) break;   // only the row's 2^L slots are used
            keys[sidx] = -1;
            if (MODE == MODE_F64) {
                dv[sidx] = 0.0;      // native FP64: one double per slot over hi|lo
            } else {
                hi[sidx] = 0.f;
                lo[sidx] = 0.f;
                lo2[sidx] = 0.f;
            }
        }
        // rows with an A value outside the double-word range accumulate natively
        bool nat = MODE == MODE_F64 || b_bad;
        // rows longer than one staging batch check their A values for the
        // double-word range first; shorter rows find out while staging
        if (MODE == MODE_DW && !nat) {
            bool ok = true;
            if (plen > E)
                for (int pp = gl; pp < plen; pp += G) dw_split(((const double *)a.aval)[p0 + pp], ok);
            const unsigned bad = __ballot_sync(0xffffffffu, !ok);
            nat = ((bad >> gbase) & lmask) != 0;
        }
        const int maxlen = __reduce_max_sync(0xffffffffu, plen);
        bool wnat = false, three = false;
        for (int pb = 0; pb < maxlen; pb += E) {
            // stage entries [pb, pb+E): lane gl takes EL consecutive entries
            int cnt[EL];
            int lsum = 0;
            bool split_ok = true;
#pragma unroll
            for (int u = 0; u < EL; u++) {
                const int e = gl * EL + u;
                const int pidx = pb + e;
                int len = 0;
                if (pidx < plen) {
                    const int k = a.acol[p0 + pidx];
                    const int4 d = bdesc[k];
                    len = d.z;
                    eq0[e] = desc_start(d);
                    const V av = ((const V *)a.aval)[p0 + pidx];
                    if (MODE == MODE_DW && !nat) {
                        const float2 s2 = dw_split((double)av, split_ok);
                        ea[e] = __longlong_as_double(((long long)__float_as_uint(s2.y) << 32) |
                                                     (long long)__float_as_uint(s2.x));
                    } else {
                        ea[e] = (double)av;
                    }
                }
                cnt[u] = len;
                lsum += len;
            }
            if (pb == 0) {
                if (MODE == MODE_DW) {
                    // a short row with a value out of range: native, staged again
                    const unsigned bad = __ballot_sync(0xffffffffu, !split_ok);
                    if (!nat && ((bad >> gbase) & lmask) != 0) {
                        nat = true;
#pragma unroll
                        for (int u = 0; u < EL; u++) {
                            const int e = gl * EL + u;
                            if (e < plen) ea[e] = ((const double *)a.aval)[p0 + e];
                        }
                    }
                }
                // warps without native rows add with atomics (three levels for
                // double-words); a warp holding a native row merges same-slot
                // lanes with __match_any_sync and adds in turns
                wnat = MODE == MODE_DW && __any_sync(0xffffffffu, nat);
                three = !wnat || plen > DW2_MAX_TERMS;
            }
            // exclusive scan of the lanes' sums within the row's group
            int incl = lsum;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d, G);
                if (gl >= d) incl += y;
            }
            int run = incl - lsum;
#pragma unroll
            for (int u = 0; u < EL; u++) {
                pre[gl * EL + u] = run;
                run += cnt[u];
            }
            if (gl == G - 1) pre[E] = incl;
            const int total = __shfl_sync(0xffffffffu, incl, gbase + G - 1);
            const int maxtot = __reduce_max_sync(0xffffffffu, total);
            __syncwarp();
            // the lane's current stored entry: its first product (pe), the
            // next entry's (pn), its start in B and its value, in registers;
            // reloaded only when the cursor moves on
            int e = 0, pe = 0, pn = pre[1];
            long long q0 = eq0[0];
            double ae = ea[0];
            for (int t0 = 0; t0 < maxtot; t0 += G) {
                const int t = t0 + gl;
                const bool valid = t < total;
                int slot = -1;
                float px = 0.f, py = 0.f;   // product payload (see acc below)
                if (valid) {
                    if (pn <= t) {
                        do {
                            e++;
                            pe = pn;
                            pn = pre[e + 1];
                        } while (pn <= t);
                        q0 = eq0[e];
                        ae = ea[e];
                    }
                    const int64_t q = q0 + (t - pe);
                    slot = map_slot(keys, L, a.bcol[q]);
                    if (slot < 0) flag |= DERR_PROBE;
                    if (MODE == MODE_F32) {
                        px = (float)ae * ((const float *)a.bval)[q];
                    } else if (MODE == MODE_DW && !nat) {
                        const unsigned long long bits = (unsigned long long)__double_as_longlong(ae);
                        const float2 a2 = make_float2(__uint_as_float((unsigned)bits),
                                                      __uint_as_float((unsigned)(bits >> 32)));
                        const float2 pr = dw_mul(a2, a.bsplit[q]);
                        px = pr.x;
                        py = pr.y;
                    } else {
                        const double pd = ae * ((const double *)a.bval)[q];
                        px = __int_as_float(__double2loint(pd));
                        py = __int_as_float(__double2hiint(pd));
                    }
                }
                if (!wnat) {
                    if (slot >= 0) {
                        if (MODE == MODE_F32) {
                            atomicAdd(&hi[slot], px);
                        } else if (MODE == MODE_F64) {
                            atomicAdd(&dv[slot], __hiloint2double(__float_as_int(py), __float_as_int(px)));
                        } else {
                            float s1, e1, tt, f, s2, e2;
                            const float o1 = atomicAdd(&hi[slot], px);
                            two_sum(o1, px, s1, e1);
                            two_sum(e1, py, tt, f);
                            const float o2 = atomicAdd(&lo[slot], tt);
                            two_sum(o2, tt, s2, e2);
                            atomicAdd(&lo2[slot], __fadd_rn(e2, f));
                        }
                    }
                    continue;
                }
                // lanes of this row holding the same slot update it in turns,
                // ordered by their rank among those lanes
                const unsigned key = slot >= 0 ? (unsigned)(rs * SMAX + slot) : 0x80000000u | lane;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const int rank = __popc(peers & ((1u << lane) - 1));
                const int maxr = __reduce_max_sync(0xffffffffu, slot >= 0 ? rank : 0);
                for (int j = 0; j <= maxr; j++) {
                    if (slot >= 0 && rank == j) acc_slot<MODE>(hi, lo, lo2, slot, nat, three, px, py);
                    __syncwarp();
                }
                __syncwarp();
            }
            __syncwarp();
        }
        // compact the occupied slots of each row to the front (read all, then
        // write); only as many slots as the warp's largest map
        const int smax_w = __reduce_max_sync(0xffffffffu, S);
        int kq[PER];
        float hq[PER], lq[PER], l2q[PER];
#pragma unroll
        for (int t = 0; t < PER; t++) {
            const int sidx = gl + t * G;
            kq[t] = -1;
            if (t * G >= smax_w) continue;
            kq[t] = sidx < S ? keys[sidx] : -1;
            if (MODE == MODE_F64) {
                const double d = dv[sidx];
                hq[t] = __int_as_float(__double2loint(d));
                lq[t] = __int_as_float(__double2hiint(d));
            } else {
                hq[t] = hi[sidx];
                lq[t] = lo[sidx];
                l2q[t] = lo2[sidx];
            }
        }
        __syncwarp();
        int cntr = 0;
#pragma unroll
        for (int t = 0; t < PER; t++) {
            if (t * G >= smax_w) break;   // warp-uniform
            const bool occ = kq[t] != -1;
            const unsigned m = (__ballot_sync(0xffffffffu, occ) >> gbase) & lmask;
            if (occ) {
                const int pos = cntr + __popc(m & ((1u << gl) - 1));
                keys[pos] = kq[t];
                if (MODE == MODE_F64) {
                    dv[pos] = __hiloint2double(__float_as_int(lq[t]), __float_as_int(hq[t]));
                } else {
                    hi[pos] = hq[t];
                    lo[pos] = lq[t];
                    lo2[pos] = l2q[t];
                }
            }
            cntr += __popc(m);
        }
        __syncwarp();
        if (active && cntr != nn) {
            flag |= DERR_COUNT;
            cntr = min(cntr, nn);
        }
        if (!active) cntr = 0;
        // rank by counting smaller keys; write each row in ascending order
        for (int e = gl; e < cntr; e += G) {
            const int key = keys[e];
            int r = 0;
            for (int u = 0; u < cntr; u++) r += keys[u] < key;
            a.ccol[out + r] = key;
            if (MODE == MODE_F32)
                ((float *)a.cval)[out + r] = hi[e];
            else if (MODE == MODE_F64)
                ((double *)a.cval)[out + r] = dv[e];
            else if (MODE == MODE_DW && !nat)
                ((double *)a.cval)[out + r] = three ? dw3_to_double(hi[e], lo[e], lo2[e])
                                                    : dw_to_double(hi[e], lo[e]);
            else
                ((double *)a.cval)[out + r] = __hiloint2double(__float_as_int(lo[e]), __float_as_int(hi[e]));
        }
        __syncwarp();
    }
    if (flag) atomicOr(err, flag);
}

// Bitonic sort of P (power of two) keys with values in shared memory by NT
// cooperating threads; sync() separates the stages.
template <typename V, typename Sync>
__device__ __forceinline__ void bitonic(int *k, V *v, int P, int tid, int NT, Sync sync) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < P / 2; t += NT) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const int x = k[lo], y = k[hi];
                if ((x > y) == asc) {
                    k[lo] = y;
                    k[hi] = x;
                    const V tv = v[lo];
                    v[lo] = v[hi];
                    v[hi] = tv;
                }
            }
            sync();
        }
    }
}

// Writes a row's n compacted entries (ck[x], cv[x]) to ccol/cval in
// ascending column order without sorting the columns: the row's distinct
// 32-column blocks are gathered in a map (block -> OR of the bit masks, the
// compression of Section 2.1 applied to the output), only the blocks are
// sorted, prefix counts of their masks give each block's first rank, and an
// entry's rank is its block's plus the number of the block's columns below
// it.  Map of 2^LB slots (bkey, bm, bb: key, mask, first rank), list of at
// most lcap blocks (lkey, lval: block, its slot).  cnt, fail: two shared
// ints.  NT threads (tid) take part; sync() orders them.  Returns false,
// with nothing written, when the blocks do not fit (more than lcap, or a
// full map): the caller then sorts the columns themselves.
template <typename Vin, typename Vout, typename Sync>
__device__ bool write_by_blocks(const int *ck, const Vin *cv, int n, int *bkey, unsigned *bm, int *bb, int LB,
                                int *lkey, int *lval, int lcap, int *cnt, int *fail, int tid, int NT, Sync sync,
                                int32_t *ccol, Vout *cval) {
    const int SB = 1 << LB;
    for (int u = tid; u < SB; u += NT) {
        bkey[u] = -1;
        bm[u] = 0u;
    }
    if (tid == 0) {
        *cnt = 0;
        *fail = 0;
    }
    sync();
    for (int x = tid; x < n; x += NT) {
        const int col = ck[x];
        if (!sym_insert(bkey, bm, LB, col >> 5, 1u << (col & 31))) *fail = 1;
    }
    sync();
    for (int u = tid; u < SB; u += NT) {
        const int k = bkey[u];
        if (k >= 0) {
            const int pos = atomicAdd(cnt, 1);
            if (pos < lcap) {
                lkey[pos] = k;
                lval[pos] = u;
            }
        }
    }
    sync();
    const int nb = *cnt;
    if (*fail || nb > lcap) return false;
    const int P = next_pow2(nb);
    for (int k = nb + tid; k < P; k += NT) {
        lkey[k] = INT_MAX;
        lval[k] = 0;
    }
    sync();
    bitonic<int>(lkey, lval, P, tid, NT, sync);
    if (tid < 32) {   // first ranks: exclusive prefix of the masks' counts, in block order
        int carry = 0;
        for (int k0 = 0; k0 < nb; k0 += 32) {
            const int k = k0 + tid;
            const int c = k < nb ? __popc(bm[lval[k]]) : 0;
            int incl = c;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (tid >= d) incl += y;
            }
            if (k < nb) bb[lval[k]] = carry + incl - c;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    sync();
    const unsigned msk = (unsigned)SB - 1;
    for (int x = tid; x < n; x += NT) {
        const int col = ck[x];
        const int blk = col >> 5;
        unsigned h = hash_slot(blk, LB);
        for (int probe = 0; probe < SB && bkey[h] != blk; probe++) h = (h + 1) & msk;
        const int r = bb[h] + __popc(bm[h] & ((1u << (col & 31)) - 1u));
        if (bkey[h] != blk || r < 0 || r >= n) continue;   // cannot happen: every block was inserted
        ccol[r] = col;
        cval[r] = (Vout)cv[x];
    }
    return true;
}

// Which dense rank accumulator takes a row of bins 3-4 (0: none, the hash
// maps of k_num_wide do): the smallest whose bitmap covers the row's span
// of 32-column blocks and whose value array holds its outputs.  Smaller
// tiers use less shared memory per warp, so more warps run per SM.
constexpr int RANK_BW1 = 512, RANK_NMAX1 = 1024, RANK_BW2 = 1024, RANK_NMAX2 = 512, RANK_BW3 = 2048,
              RANK_NMAX3 = 1024;
__device__ __forceinline__ int rank_tier(int span, int nn) {
    if (span <= 0) return 0;
    if (span <= RANK_BW1 && nn <= RANK_NMAX1) return 1;
    if (span <= RANK_BW2 && nn <= RANK_NMAX2) return 2;
    if (span <= RANK_BW3 && nn <= RANK_NMAX3) return 3;
    return 0;
}

// Rows of bins 2-4 whose columns fall within 32*BW consecutive columns: a
// dense accumulator over the row's column span (the dense accumulator of
// Section 3.1, restricted to the span and held in shared memory).  Pass 1
// marks every reachable column in a bitmap over the span; prefix counts of
// the bitmap words turn a column into its rank in the output row; pass 2
// adds every product into vals[rank] (atomically: FP32 and native FP64 in
// their type, double-words through the three-level dw_atomic_acc).  The row
// is then written in column order straight from the bitmap: no hash map,
// no sort.  Products are dealt out over the warp's 32 lanes as in the other
// kernels.  Per warp: bitmap, 16-bit prefix counts, NMAX values.
template <int MODE>
struct RankVal {
    static constexpr int bytes = MODE == MODE_F32 ? 4 : (MODE == MODE_DW ? 12 : 8);
};

constexpr int RANK_U = 4;   // products per lane per step in the rank kernels

template <int BW, int NMAX, int WPB, int MODE>
struct RankLayout {
    static constexpr size_t per_warp =
        ((size_t)BW * 6 + (size_t)BW / 8 + (size_t)NMAX * RankVal<MODE>::bytes + 32 * 16 + 33 * 4 + 64 + 15) &
        ~(size_t)15;
    static constexpr size_t bytes = per_warp * WPB;
};

// The bitmap words a row touches are listed by a summary bitmap (one bit
// per word), so the prefix counts, the output and the clean-up visit only
// those words: the work per row follows its outputs, not its span.  A row
// leaves its bitmap words and summary zero for the next.
template <int BW, int NMAX, int WPB, int MODE>
__global__ void __launch_bounds__(WPB * 32, 1) k_num_rank(NumP a, const int4 *__restrict__ bdesc,
                                                       const int2 *__restrict__ spans,
                                                       const int32_t *__restrict__ rows, int64_t count,
                                                       int tier, const DevState *st, int *err) {
    using Lay = RankLayout<BW, NMAX, WPB, MODE>;
    using V = ValT<MODE>;
    constexpr int E = 32, NS = BW / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + (size_t)w * Lay::per_warp;
    long long *eq0 = (long long *)base;
    double *ea = (double *)(eq0 + E);
    unsigned *bits = (unsigned *)(ea + E);
    unsigned *summ = bits + BW;
    unsigned short *pref = (unsigned short *)(summ + NS);
    unsigned char *vbase = (unsigned char *)(((uintptr_t)(pref + BW) + 15) & ~(uintptr_t)15);
    float *vf = (float *)vbase;                              // FP32
    double *v8 = (double *)vbase;                            // native FP64
    float2 *v2 = (float2 *)vbase;                            // double-word hi, lo
    float *v3 = (float *)(v2 + NMAX);                        // third level
    int *pre = (int *)(vbase + (size_t)NMAX * RankVal<MODE>::bytes);
    const bool b_bad = MODE == MODE_DW && st->b_out_of_range;
    int flag = 0;
    for (int x = lane; x < BW; x += 32) bits[x] = 0;
    for (int x = lane; x < NS; x += 32) summ[x] = 0;
    __syncwarp();
    for (int64_t t = (int64_t)blockIdx.x * WPB + w; t < count; t += (int64_t)gridDim.x * WPB) {
        const int i = rows[t];
        const int64_t out = a.crp[i];
        const int nn = (int)(a.crp[i + 1] - out);
        if (nn > NMAX) continue;
        const int2 sp = spans[t];
        const int bmin = sp.x, nw = sp.y;
        if (nw > BW || nw == 0 || rank_tier(nw, nn) != tier) continue;
        const int64_t p0 = a.arp[i];
        const int plen = (int)(a.arp[i + 1] - p0);
        bool nat = MODE == MODE_F64 || b_bad;
        if (MODE == MODE_DW && !nat) {
            bool ok = true;
            for (int pp = lane; pp < plen; pp += 32) dw_split(((const double *)a.aval)[p0 + pp], ok);
            nat = !__all_sync(0xffffffffu, ok);
        }
        for (int x = lane; x < nn; x += 32) {
            if (MODE == MODE_F32) vf[x] = 0.f;
            else if (MODE == MODE_DW) { v2[x] = make_float2(0.f, 0.f); v3[x] = 0.f; }
            else v8[x] = 0.0;
        }
        const int ns = (nw + 31) / 32;                 // summary words of the span
        const int sper = (ns + 31) / 32;               // per lane, contiguous
        const int s0 = min(ns, lane * sper), s1 = min(ns, s0 + sper);
        __syncwarp();
        // a row whose stored a_ik fit one batch is staged once, for both passes
        bool staged = false;
        int total1 = 0;
        for (int pass = 0; pass < 2; pass++) {
            for (int pb = 0; pb < plen; pb += E) {
                int total;
                if (pass == 1 && staged) {
                    total = total1;
                } else {
                    int len = 0;
                    if (pb + lane < plen) {
                        const int4 d = bdesc[a.acol[p0 + pb + lane]];
                        len = d.z;
                        eq0[lane] = desc_start(d);
                        const V av = ((const V *)a.aval)[p0 + pb + lane];
                        if (MODE == MODE_DW && !nat) {
                            bool dummy = true;
                            const float2 s2 = dw_split((double)av, dummy);
                            ea[lane] = __longlong_as_double(((long long)__float_as_uint(s2.y) << 32) |
                                                            (long long)__float_as_uint(s2.x));
                        } else {
                            ea[lane] = (double)av;
                        }
                    }
                    int incl = len;
                    for (int d = 1; d < 32; d <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, d);
                        if (lane >= d) incl += y;
                    }
                    pre[lane] = incl - len;
                    if (lane == 31) pre[E] = incl;
                    total = __shfl_sync(0xffffffffu, incl, 31);
                    if (pass == 0 && plen <= E) {
                        staged = true;
                        total1 = total;
                    }
                    __syncwarp();
                }
                // RANK_U products per lane per step (t, t + 32, ...): their
                // loads of B are issued together, so a row waits for the
                // memory once per step, not once per product
                int e = 0;
                for (int t0 = 0; t0 < total; t0 += 32 * RANK_U) {
                    int ee[RANK_U], cc[RANK_U];
                    int64_t qq[RANK_U];
#pragma unroll
                    for (int u = 0; u < RANK_U; u++) {
                        const int tt = t0 + u * 32 + lane;
                        ee[u] = -1;
                        qq[u] = 0;
                        if (tt < total) {
                            while (pre[e + 1] <= tt) e++;
                            ee[u] = e;
                            qq[u] = eq0[e] + (tt - pre[e]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < RANK_U; u++) cc[u] = ee[u] >= 0 ? a.bcol[qq[u]] : 0;
                    if (pass == 0) {
#pragma unroll
                        for (int u = 0; u < RANK_U; u++) {
                            if (ee[u] < 0) continue;
                            const int col = cc[u];
                            const int wd = (col >> 5) - bmin;
                            if (atomicOr(&bits[wd], 1u << (col & 31)) == 0)
                                atomicOr(&summ[wd >> 5], 1u << (wd & 31));
                        }
                    } else if (MODE == MODE_F32) {
                        float bv[RANK_U];
#pragma unroll
                        for (int u = 0; u < RANK_U; u++) bv[u] = ee[u] >= 0 ? ((const float *)a.bval)[qq[u]] : 0.f;
#pragma unroll
                        for (int u = 0; u < RANK_U; u++) {
                            if (ee[u] < 0) continue;
                            const int col = cc[u];
                            const int wd = (col >> 5) - bmin;
                            const int r = (int)pref[wd] + __popc(bits[wd] & ((1u << (col & 31)) - 1));
                            atomicAdd(&vf[r], (float)ea[ee[u]] * bv[u]);
                        }
                    } else if (MODE == MODE_DW && !nat) {
                        float2 bv[RANK_U];
#pragma unroll
                        for (int u = 0; u < RANK_U; u++) bv[u] = ee[u] >= 0 ? a.bsplit[qq[u]] : make_float2(0.f, 0.f);
#pragma unroll
                        for (int u = 0; u < RANK_U; u++) {
                            if (ee[u] < 0) continue;
                            const int col = cc[u];
                            const int wd = (col >> 5) - bmin;
                            const int r = (int)pref[wd] + __popc(bits[wd] & ((1u << (col & 31)) - 1));
                            const unsigned long long bb = (unsigned long long)__double_as_longlong(ea[ee[u]]);
                            const float2 a2 = make_float2(__uint_as_float((unsigned)bb),
                                                          __uint_as_float((unsigned)(bb >> 32)));
                            dw_atomic_acc(v2, v3, r, dw_mul(a2, bv[u]));
                        }
                    } else {
                        double bv[RANK_U];
#pragma unroll
                        for (int u = 0; u < RANK_U; u++) bv[u] = ee[u] >= 0 ? ((const double *)a.bval)[qq[u]] : 0.0;
#pragma unroll
                        for (int u = 0; u < RANK_U; u++) {
                            if (ee[u] < 0) continue;
                            const int col = cc[u];
                            const int wd = (col >> 5) - bmin;
                            const int r = (int)pref[wd] + __popc(bits[wd] & ((1u << (col & 31)) - 1));
                            atomicAdd(&v8[r], ea[ee[u]] * bv[u]);
                        }
                    }
                }
                __syncwarp();
            }
            if (pass == 0) {
                // prefix counts of the touched words, in word order
                int sum = 0;
                for (int y = s0; y < s1; y++) {
                    unsigned sw = summ[y];
                    while (sw) {
                        const int x = y * 32 + __ffs(sw) - 1;
                        sw &= sw - 1;
                        sum += __popc(bits[x]);
                    }
                }
                int incl = sum;
                for (int d = 1; d < 32; d <<= 1) {
                    const int yv = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += yv;
                }
                int run = incl - sum;
                for (int y = s0; y < s1; y++) {
                    unsigned sw = summ[y];
                    while (sw) {
                        const int x = y * 32 + __ffs(sw) - 1;
                        sw &= sw - 1;
                        pref[x] = (unsigned short)run;
                        run += __popc(bits[x]);
                    }
                }
                if (__shfl_sync(0xffffffffu, incl, 31) != nn) flag |= DERR_COUNT;
                __syncwarp();
            }
        }
        // write the row in column order from the touched words, clearing them
        for (int y = s0; y < s1; y++) {
            unsigned sw = summ[y];
            while (sw) {
                const int x = y * 32 + __ffs(sw) - 1;
                sw &= sw - 1;
                unsigned word = bits[x];
                int r = pref[x];
                while (word) {
                    const int b = __ffs(word) - 1;
                    word &= word - 1;
                    if (r < nn) {
                        a.ccol[out + r] = (bmin + x) * 32 + b;
                        if (MODE == MODE_F32) ((float *)a.cval)[out + r] = vf[r];
                        else if (MODE == MODE_DW && !nat) ((double *)a.cval)[out + r] = dw3_to_double(v2[r].x, v2[r].y, v3[r]);
                        else ((double *)a.cval)[out + r] = v8[r];
                    }
                    r++;
                }
                bits[x] = 0;
            }
            summ[y] = 0;
        }
        __syncwarp();
    }
    if (flag) atomicOr(err, flag);
}

// Bins 3-4 (and bin 2 when the small-row cap is 16): a warp per listed row,
// a map of up to SMAX slots (rows with at most SMAX/2 outputs).  The row's
// products are dealt out over the 32 lanes as in k_num_small (stored a_ik
// staged 32 at a time with the prefix sums of nnz(B_k)); slots are updated
// atomically (FP32 and native FP64 in their type, double-words through the
// three-level dw_atomic_acc).  The output is written in column order
// without a sort when the row's column span is at most 32*BW: the columns
// are marked in a bitmap over the span, each lane walks a run of its words
// from its prefix count and looks the values up in the map.  Wider rows
// are compacted and sorted with a bitonic network.
template <int MODE>
struct WideSlot {   // bytes per map slot: key + value (+ third level); 16 in
    // every mode, so that the output ordering by blocks (4 ints per slot)
    // can reuse the map's space
    static constexpr int bytes = 16;
};

template <int SMAX, int BW, int WPB, int MODE>
struct WideLayout {
    static constexpr size_t table = (size_t)SMAX * WideSlot<MODE>::bytes;
    static constexpr size_t aux = ((size_t)BW * 4 > (size_t)SMAX / 2 * 12 ? (size_t)BW * 4 : (size_t)SMAX / 2 * 12);
    static constexpr size_t stage = 32 * 16 + 33 * 4 + 16;
    static constexpr size_t per_warp = (table + aux + stage + 15) & ~(size_t)15;
    static constexpr size_t bytes = per_warp * WPB;
};

template <int SMAX, int BW, int WPB, int MODE>
__global__ void __launch_bounds__(WPB * 32, 1) k_num_wide(NumP a, const int4 *__restrict__ bdesc,
                                                       const int2 *__restrict__ spans,
                                                       const int32_t *__restrict__ rows, int64_t count,
                                                       int min_nnz, int min_span_words, const DevState *st,
                                                       int *err) {
    using Lay = WideLayout<SMAX, BW, WPB, MODE>;
    using V = ValT<MODE>;
    constexpr int E = 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + (size_t)w * Lay::per_warp;
    // table: FP32 {float val}[S] | keys[S];  otherwise {float2 or double}[S] | lo2[S] | keys[S]
    float2 *v2 = (float2 *)base;
    double *v8 = (double *)base;
    float *vf = (float *)base;
    float *v3 = MODE == MODE_F32 ? nullptr : (float *)(v8 + SMAX);
    int *keys = MODE == MODE_F32 ? (int *)(vf + SMAX) : (int *)(v3 + SMAX);
    unsigned *bits = (unsigned *)(base + Lay::table);
    int *ck = (int *)bits;
    double *cv = (double *)((int *)bits + SMAX / 2);
    long long *eq0 = (long long *)(base + Lay::table + Lay::aux);
    double *ea = (double *)(eq0 + E);
    int *pre = (int *)(ea + E);
    int *ncount = pre + E + 1;
    const bool b_bad = MODE == MODE_DW && st->b_out_of_range;
    int flag = 0;
    for (int64_t t = (int64_t)blockIdx.x * WPB + w; t < count; t += (int64_t)gridDim.x * WPB) {
        const int i = rows[t];
        const int64_t out = a.crp[i];
        const int nn = (int)(a.crp[i + 1] - out);
        if (nn < min_nnz || nn > SMAX / 2) continue;
        if (min_span_words > 0 && rank_tier(spans[t].y, nn) != 0) continue;
        int S = next_pow2(2 * nn);
        S = S < 32 ? 32 : (S > SMAX ? SMAX : S);
        const int L = __ffs(S) - 1;
        for (int u = lane; u < S; u += 32) {
            keys[u] = -1;
            if (MODE == MODE_F32) {
                vf[u] = 0.f;
            } else {
                v8[u] = 0.0;
                v3[u] = 0.f;
            }
        }
        const int64_t p0 = a.arp[i];
        const int plen = (int)(a.arp[i + 1] - p0);
        bool nat = MODE == MODE_F64 || b_bad;
        if (MODE == MODE_DW && !nat) {
            bool ok = true;
            for (int pp = lane; pp < plen; pp += 32) dw_split(((const double *)a.aval)[p0 + pp], ok);
            nat = !__all_sync(0xffffffffu, ok);
        }
        int cmin = INT_MAX, cmax = -1;
        __syncwarp();
        for (int pb = 0; pb < plen; pb += E) {
            int len = 0;
            if (pb + lane < plen) {
                const int4 d = bdesc[a.acol[p0 + pb + lane]];
                len = d.z;
                eq0[lane] = desc_start(d);
                const V av = ((const V *)a.aval)[p0 + pb + lane];
                if (MODE == MODE_DW && !nat) {
                    bool dummy = true;
                    const float2 s2 = dw_split((double)av, dummy);
                    ea[lane] = __longlong_as_double(((long long)__float_as_uint(s2.y) << 32) |
                                                    (long long)__float_as_uint(s2.x));
                } else {
                    ea[lane] = (double)av;
                }
            }
            int incl = len;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            pre[lane] = incl - len;
            if (lane == 31) pre[E] = incl;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            int e = 0;
            const bool f64 = MODE == MODE_F64 || (MODE == MODE_DW && nat);   // uniform in the warp
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int tt = t0 + lane;
                int slot = -1;
                double pv = 0.0;
                if (tt < total) {
                    while (pre[e + 1] <= tt) e++;
                    const int64_t q = eq0[e] + (tt - pre[e]);
                    const int col = a.bcol[q];
                    cmin = min(cmin, col);
                    cmax = max(cmax, col);
                    slot = map_slot(keys, L, col);
                    if (slot < 0) {
                        flag |= DERR_PROBE;
                    } else if (MODE == MODE_F32) {
                        atomicAdd(&vf[slot], (float)ea[e] * ((const float *)a.bval)[q]);
                    } else if (MODE == MODE_DW && !nat) {
                        const unsigned long long bb = (unsigned long long)__double_as_longlong(ea[e]);
                        const float2 a2 = make_float2(__uint_as_float((unsigned)bb), __uint_as_float((unsigned)(bb >> 32)));
                        dw_atomic_acc(v2, v3, slot, dw_mul(a2, a.bsplit[q]));
                    } else {
                        pv = ea[e] * ((const double *)a.bval)[q];
                    }
                }
                if (f64) warp_acc_f64(v8, slot, slot >= 0, pv, lane);
            }
            __syncwarp();
        }
        for (int d = 16; d > 0; d >>= 1) {
            cmin = min(cmin, __shfl_xor_sync(0xffffffffu, cmin, d));
            cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, d));
        }
        const int64_t span = cmax >= cmin ? (int64_t)cmax - cmin + 1 : 0;
        auto slot_value = [&](int u) -> double {
            if (MODE == MODE_F32) return (double)vf[u];
            if (MODE == MODE_DW && !nat) return dw3_to_double(v2[u].x, v2[u].y, v3[u]);
            return v8[u];
        };
        if (span <= 32LL * BW) {
            const int nw = (int)((span + 31) >> 5);
            for (int x = lane; x < nw; x += 32) bits[x] = 0;
            __syncwarp();
            for (int u = lane; u < S; u += 32) {
                const int key = keys[u];
                if (key >= 0) atomicOr(&bits[(key - cmin) >> 5], 1u << ((key - cmin) & 31));
            }
            __syncwarp();
            const int per = (nw + 31) / 32;
            const int x0 = min(nw, lane * per), x1 = min(nw, x0 + per);
            int sum = 0;
            for (int x = x0; x < x1; x++) sum += __popc(bits[x]);
            int incl = sum;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            if (__shfl_sync(0xffffffffu, incl, 31) != nn) flag |= DERR_COUNT;
            int r = incl - sum;
            for (int x = x0; x < x1; x++) {
                unsigned word = bits[x];
                while (word) {
                    const int bpos = __ffs(word) - 1;
                    word &= word - 1;
                    const int col = cmin + x * 32 + bpos;
                    unsigned hh = hash_slot(col, L);
                    while (keys[hh] != col) hh = (hh + 1) & (S - 1);
                    if (r < nn) {
                        a.ccol[out + r] = col;
                        if (MODE == MODE_F32) ((float *)a.cval)[out + r] = vf[hh];
                        else ((double *)a.cval)[out + r] = slot_value((int)hh);
                    }
                    r++;
                }
            }
        } else {
            // compact (values as double), bitonic sort, write
            if (lane == 0) *ncount = 0;
            __syncwarp();
            for (int u0 = 0; u0 < S; u0 += 32) {
                const int u = u0 + lane;
                const int key = keys[u];
                const bool occ = key >= 0;
                const unsigned m = __ballot_sync(0xffffffffu, occ);
                const int basec = *ncount;
                if (occ) {
                    const int pos = basec + __popc(m & ((1u << lane) - 1));
                    if (pos < SMAX / 2) {
                        ck[pos] = key;
                        cv[pos] = slot_value(u);
                    }
                }
                __syncwarp();
                if (lane == 0) *ncount = basec + __popc(m);
                __syncwarp();
            }
            int n = min(*ncount, SMAX / 2);
            if (n != nn) {
                flag |= DERR_COUNT;
                n = min(n, nn);
            }
            // the map's slots are free now: order the output by its blocks
            using Vout = typename std::conditional<MODE == MODE_F32, float, double>::type;
            int SB = next_pow2(2 * n);
            SB = SB < 32 ? 32 : SB;
            int *tb = (int *)base;
            const bool done = write_by_blocks<double, Vout>(
                ck, cv, n, tb, (unsigned *)(tb + SB), tb + 2 * SB, __ffs(SB) - 1, tb + 3 * SB,
                tb + 3 * SB + SB / 2, SB / 2, ncount, pre, lane, 32, [] { __syncwarp(); }, a.ccol + out,
                (Vout *)a.cval + out);
            __syncwarp();
            if (!done) {
                const int P = next_pow2(n);
                for (int x = n + lane; x < P; x += 32) ck[x] = INT_MAX;
                __syncwarp();
                bitonic<double>(ck, cv, P, lane, 32, [] { __syncwarp(); });
                for (int x = lane; x < n; x += 32) {
                    a.ccol[out + x] = ck[x];
                    if (MODE == MODE_F32) ((float *)a.cval)[out + x] = (float)cv[x];
                    else ((double *)a.cval)[out + x] = cv[x];
                }
            }
        }
        __syncwarp();
    }
    if (flag) atomicOr(err, flag);
}

// ------------------------------------------------------------------ block kernels
// Insert (col, v) with atomic accumulation into a map of 2^L slots; false
// when `limit` probes found neither the key nor a free slot.
template <typename V>
__device__ __forceinline__ bool map_add(int *keys, V *vals, int L, int limit, int col, V v) {
    const unsigned msk = (1u << L) - 1;
    unsigned h = hash_slot(col, L);
#pragma unroll 1
    for (int probe = 0; probe < limit; probe++) {
        int k = ((volatile int *)keys)[h];
        if (k == col) {
            atomicAdd(&vals[h], v);
            return true;
        }
        if (k == -1) {
            int old = atomicCAS(&keys[h], -1, col);
            if (old == -1 || old == col) {
                atomicAdd(&vals[h], v);
                return true;
            }
        }
        h = (h + 1) & msk;
    }
    return false;
}

// Slots of the block map that orders a block kernel's output (at most
// BLOCK_TAB / 2 distinct 32-column blocks per row; rows with more are sorted
// by columns).
constexpr int BLOCK_TAB = 2048;

// Bins 4-5: a block per listed row, map of S slots in shared memory; warps
// take stored a_ik in turn and their lanes walk B_k; atomic accumulation in
// the value type (FP64 rows accumulate natively).
template <int BS, int S, typename V>
__global__ void __launch_bounds__(BS) k_num_block(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol, const V *__restrict__ aval,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, const V *__restrict__ bval,
    const int64_t *__restrict__ crp, int32_t *__restrict__ ccol, V *__restrict__ cval,
    const int32_t *__restrict__ rows, int64_t count, int *err) {
    constexpr int L = __builtin_ctz(S);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *vals = (V *)smem_raw;
    V *cv = vals + S;
    int *keys = (int *)(cv + S / 2);
    int *ck = keys + S;
    int *btab = ck + S / 2;   // 4 * BLOCK_TAB ints: block map and list
    __shared__ int nsh, bcnt, bfail;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int flag = 0;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        for (int s = threadIdx.x; s < S; s += BS) {
            keys[s] = -1;
            vals[s] = V(0);
        }
        if (threadIdx.x == 0) nsh = 0;
        __syncthreads();
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += BS / 32) {
            const int k = acol[p];
            const V av = aval[p];
            const int64_t q1 = brp[k + 1];
            for (int64_t q = brp[k] + lane; q < q1; q += 32)
                if (!map_add<V>(keys, vals, L, S, bcol[q], av * bval[q])) flag |= DERR_PROBE;
        }
        __syncthreads();
        for (int s = threadIdx.x; s < S; s += BS) {
            const int key = keys[s];
            const bool occ = key != -1;
            const unsigned m = __ballot_sync(0xffffffffu, occ);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&nsh, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (occ) {
                const int pos = base + __popc(m & ((1u << lane) - 1));
                if (pos < S / 2) {
                    ck[pos] = key;
                    cv[pos] = vals[s];
                }
            }
        }
        __syncthreads();
        int n = nsh;
        const int64_t out = crp[i];
        const int expect = (int)(crp[i + 1] - out);
        if (n != expect) {
            flag |= DERR_COUNT;
            n = min(min(n, expect), S / 2);
        }
        // order the output by its blocks (a map of BLOCK_TAB slots after the
        // column map); sort the columns themselves if they span too many
        const bool done = write_by_blocks<V, V>(ck, cv, n, btab, (unsigned *)(btab + BLOCK_TAB),
                                                btab + 2 * BLOCK_TAB, __builtin_ctz(BLOCK_TAB),
                                                btab + 3 * BLOCK_TAB, btab + 3 * BLOCK_TAB + BLOCK_TAB / 2,
                                                BLOCK_TAB / 2, &bcnt, &bfail, threadIdx.x, BS,
                                                [] { __syncthreads(); }, ccol + out, cval + out);
        __syncthreads();
        if (!done) {
            const int P = next_pow2(n);
            for (int e = n + threadIdx.x; e < P; e += BS) ck[e] = INT_MAX;
            __syncthreads();
            bitonic<V>(ck, cv, P, threadIdx.x, BS, [] { __syncthreads(); });
            for (int e = threadIdx.x; e < n; e += BS) {
                ccol[out + e] = ck[e];
                cval[out + e] = cv[e];
            }
        }
        __syncthreads();
    }
    if (flag) atomicOr(err, flag);
}

// Bin 6: first-level map in shared memory (bounded probing), second level in
// global memory sized for the row (Section 3.3); the row's columns are then
// marked in a bitmap whose word prefix counts give each entry its rank.
// Global memory per block: L2 keys/values (l2cap slots), bitmap and prefix
// (nwords words each); every row clears the L2 slots it uses.
constexpr int HUGE_BS = 512, HUGE_L1 = 4096, HUGE_PROBES = 16;

template <typename V>
__global__ void __launch_bounds__(HUGE_BS, 1) k_num_huge(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol, const V *__restrict__ aval,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, const V *__restrict__ bval,
    const int64_t *__restrict__ crp, int32_t *__restrict__ ccol, V *__restrict__ cval,
    const int32_t *__restrict__ rows, int64_t count, int *err, int64_t l2cap, int64_t nwords,
    unsigned char *gws) {
    constexpr int L1 = __builtin_ctz(HUGE_L1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *vals = (V *)smem_raw;
    int *keys = (int *)(vals + HUGE_L1);
    __shared__ int cmin, cmax;
    __shared__ long long red[HUGE_BS / 32];
    const size_t per_block = (size_t)l2cap * (4 + sizeof(V)) + (size_t)nwords * 8;
    unsigned char *mine = gws + per_block * blockIdx.x;
    V *g_vals = (V *)mine;
    int *g_keys = (int *)(g_vals + l2cap);
    unsigned *bits = (unsigned *)(g_keys + l2cap);
    unsigned *pref = bits + nwords;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int flag = 0;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        const int64_t out = crp[i];
        const int64_t expect = crp[i + 1] - out;
        int L2 = 1;
        while ((1LL << L2) < 2 * expect) L2++;
        for (int s = threadIdx.x; s < HUGE_L1; s += HUGE_BS) {
            keys[s] = -1;
            vals[s] = V(0);
        }
        for (int64_t s = threadIdx.x; s < (1LL << L2); s += HUGE_BS) {
            g_keys[s] = -1;
            g_vals[s] = V(0);
        }
        if (threadIdx.x == 0) {
            cmin = INT_MAX;
            cmax = -1;
        }
        __syncthreads();
        int lmin = INT_MAX, lmax = -1;
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += HUGE_BS / 32) {
            const int k = acol[p];
            const V av = aval[p];
            const int64_t q1 = brp[k + 1];
            for (int64_t q = brp[k] + lane; q < q1; q += 32) {
                const int c = bcol[q];
                const V v = av * bval[q];
                lmin = min(lmin, c);
                lmax = max(lmax, c);
                if (!map_add<V>(keys, vals, L1, HUGE_PROBES, c, v))
                    if (!map_add<V>(g_keys, g_vals, L2, 1 << L2, c, v)) flag |= DERR_PROBE;
            }
        }
        atomicMin(&cmin, lmin);
        atomicMax(&cmax, lmax);
        __syncthreads();
        for (int s = threadIdx.x; s < HUGE_L1; s += HUGE_BS) {
            const int key = keys[s];
            if (key != -1)
                if (!map_add<V>(g_keys, g_vals, L2, 1 << L2, key, vals[s])) flag |= DERR_PROBE;
        }
        const int64_t w0 = (cmax >= 0) ? (cmin >> 5) : 0;
        const int64_t w1 = (cmax >= 0) ? (cmax >> 5) + 1 : 0;
        for (int64_t x = w0 + threadIdx.x; x < w1; x += HUGE_BS) bits[x] = 0;
        __syncthreads();
        const int64_t slots = 1LL << L2;
        for (int64_t s = threadIdx.x; s < slots; s += HUGE_BS) {
            const int key = g_keys[s];
            if (key != -1) atomicOr(&bits[key >> 5], 1u << (key & 31));
        }
        __syncthreads();
        // word prefix: a contiguous chunk per thread, block scan of chunk sums
        const int64_t nw = w1 - w0;
        const int64_t chunk = (nw + HUGE_BS - 1) / HUGE_BS;
        const int64_t c0 = w0 + threadIdx.x * chunk;
        const int64_t c1 = min(w1, c0 + chunk);
        long long sum = 0;
        for (int64_t x = c0; x < c1; x++) sum += __popc(bits[x]);
        long long incl = sum;
        for (int d = 1; d < 32; d <<= 1) {
            const long long tt = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += tt;
        }
        if (lane == 31) red[w] = incl;
        __syncthreads();
        if (w == 0) {
            const long long v = lane < HUGE_BS / 32 ? red[lane] : 0;
            long long vi = v;
            for (int d = 1; d < 32; d <<= 1) {
                const long long tt = __shfl_up_sync(0xffffffffu, vi, d);
                if (lane >= d) vi += tt;
            }
            if (lane < HUGE_BS / 32) red[lane] = vi - v;
        }
        __syncthreads();
        long long run = red[w] + incl - sum;
        for (int64_t x = c0; x < c1; x++) {
            pref[x] = (unsigned)run;
            run += __popc(bits[x]);
        }
        __syncthreads();
        for (int64_t s = threadIdx.x; s < slots; s += HUGE_BS) {
            const int key = g_keys[s];
            if (key != -1) {
                const int64_t x = key >> 5;
                const int64_t r = (int64_t)pref[x] + __popc(bits[x] & ((1u << (key & 31)) - 1));
                if (r < expect) {
                    ccol[out + r] = key;
                    cval[out + r] = g_vals[s];
                } else {
                    flag |= DERR_COUNT;
                }
            }
        }
        __syncthreads();
    }
    if (flag) atomicOr(err, flag);
}

// Bin 6 when every row of B is sorted: a dense accumulator over windows of
// W columns (Section 3.1's dense accumulator, kept in shared memory a window
// at a time).  Each stored a_ik keeps a cursor into B_k and the column it
// points at.  For a window, a thread per a_ik whose next column falls in
// the window adds a_ik * b_kj into win[j - w0] (atomically) while marking j
// in a bitmap, until B_k leaves the window; rows of B longer than WIN_LONG
// are walked by whole warps instead (32 entries per step), each warp taking
// the next such a_ik from a shared counter so the window's work stays
// balanced.  The window's entries then leave in column order: prefix counts
// of the bitmap words give each its place, and the slot is cleared as it is
// read.  Windows between the row's first and last reachable column are
// visited in order, so the row is written sorted without a sort.  Global memory per block: a cursor,
// a next column and a list slot per stored entry of the longest row.
constexpr int WIN_BS = 256, WIN_BPSM = 6, WIN_LONG = 256;

template <typename V, int W>
__global__ void __launch_bounds__(WIN_BS, WIN_BPSM) k_num_window(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol, const V *__restrict__ aval,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, const V *__restrict__ bval,
    const int64_t *__restrict__ crp, int32_t *__restrict__ ccol, V *__restrict__ cval,
    const int32_t *__restrict__ rows, int64_t count, int *err, int64_t max_alen, unsigned char *gws) {
    constexpr int NW = W / 32, NWARP = WIN_BS / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *win = (V *)smem_raw;
    unsigned *bits = (unsigned *)(win + W);
    __shared__ int bmin_s, bmax_s, wtot, nlong, lnext;
    __shared__ int red[NWARP];
    const size_t per = (size_t)max_alen;
    int64_t *cpos = (int64_t *)gws + (size_t)blockIdx.x * per;
    int32_t *cnext = (int32_t *)((int64_t *)gws + (size_t)gridDim.x * per) + (size_t)blockIdx.x * per;
    int32_t *llist = (int32_t *)((int64_t *)gws + (size_t)gridDim.x * per) + (size_t)gridDim.x * per +
                     (size_t)blockIdx.x * per;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int flag = 0;
    for (int x = threadIdx.x; x < W; x += WIN_BS) win[x] = V(0);
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        const int64_t p0 = arp[i], plen = arp[i + 1] - p0;
        const int64_t out = crp[i], expect = crp[i + 1] - out;
        if (threadIdx.x == 0) {
            bmin_s = INT_MAX;
            bmax_s = -1;
            nlong = 0;
        }
        __syncthreads();
        int lmin = INT_MAX, lmax = -1;
        for (int64_t p = threadIdx.x; p < plen; p += WIN_BS) {
            const int k = acol[p0 + p];
            const int64_t q0 = brp[k], q1 = brp[k + 1];
            cpos[p] = q0;
            int nxt = INT_MAX;
            if (q1 > q0) {
                nxt = bcol[q0];
                lmin = min(lmin, nxt);
                lmax = max(lmax, bcol[q1 - 1]);
            }
            if (q1 - q0 > WIN_LONG) {
                llist[atomicAdd(&nlong, 1)] = (int)p;
                nxt = INT_MAX;   // walked by warps
            }
            cnext[p] = nxt;
        }
        atomicMin(&bmin_s, lmin);
        atomicMax(&bmax_s, lmax);
        __syncthreads();
        const int cmin = bmin_s, cmax = bmax_s, nl = nlong;
        int64_t written = 0;
        for (int64_t w0 = cmax >= 0 ? ((int64_t)cmin / W) * W : 1; w0 <= cmax; w0 += W) {
            const int64_t w1 = w0 + W;
            for (int x = threadIdx.x; x < NW; x += WIN_BS) bits[x] = 0;
            if (threadIdx.x == 0) lnext = 0;
            __syncthreads();
            // short rows of B: a thread per stored a_ik
            for (int64_t p = threadIdx.x; p < plen; p += WIN_BS) {
                int c = cnext[p];
                if (c == INT_MAX || (int64_t)c >= w1) continue;   // INT_MAX: done or long
                const int k = acol[p0 + p];
                const V av = aval[p0 + p];
                const int64_t q1 = brp[k + 1];
                int64_t q = cpos[p];
                while (true) {
                    const int rel = (int)(c - w0);
                    atomicAdd(&win[rel], av * bval[q]);
                    atomicOr(&bits[rel >> 5], 1u << (rel & 31));
                    if (++q >= q1) { c = INT_MAX; break; }
                    c = bcol[q];
                    if ((int64_t)c >= w1) break;
                }
                cpos[p] = q;
                cnext[p] = c;
            }
            // long rows of B: a warp per stored a_ik, 32 entries per step; warps
            // take the next a_ik from a shared counter so that the window's
            // work is balanced across them
            while (true) {
                int j = 0;
                if (lane == 0) j = atomicAdd(&lnext, 1);
                j = __shfl_sync(0xffffffffu, j, 0);
                if (j >= nl) break;
                const int p = llist[j];
                const int k = acol[p0 + p];
                const V av = aval[p0 + p];
                int64_t c = cpos[p];
                const int64_t q1 = brp[k + 1];
                while (c < q1) {
                    const int64_t q = c + lane;
                    const int col = q < q1 ? bcol[q] : INT_MAX;
                    const bool in = col < w1;
                    const unsigned m = __ballot_sync(0xffffffffu, in);
                    if (in) {
                        const int rel = (int)(col - w0);
                        atomicAdd(&win[rel], av * bval[q]);
                        atomicOr(&bits[rel >> 5], 1u << (rel & 31));
                    }
                    c += __popc(m);
                    if (m != 0xffffffffu) break;
                }
                if (lane == 0) cpos[p] = c;
            }
            __syncthreads();
            // prefix counts of the words
            constexpr int PERT = (NW + WIN_BS - 1) / WIN_BS;
            int sum = 0;
#pragma unroll
            for (int u = 0; u < PERT; u++) {
                const int x = threadIdx.x * PERT + u;
                if (x < NW) sum += __popc(bits[x]);
            }
            int incl = sum;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            if (lane == 31) red[w] = incl;
            __syncthreads();
            if (w == 0) {
                const int v = lane < NWARP ? red[lane] : 0;
                int vi = v;
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, vi, d);
                    if (lane >= d) vi += y;
                }
                if (lane < NWARP) red[lane] = vi - v;
                if (lane == NWARP - 1) wtot = vi;
            }
            __syncthreads();
            // emit this thread's words in column order, clearing the slots read
            int64_t r = written + red[w] + incl - sum;
#pragma unroll
            for (int u = 0; u < PERT; u++) {
                const int x = threadIdx.x * PERT + u;
                if (x >= NW) continue;
                unsigned word = bits[x];
                while (word) {
                    const int b = __ffs(word) - 1;
                    word &= word - 1;
                    const int idx = x * 32 + b;
                    if (r < expect) {
                        ccol[out + r] = (int)(w0 + idx);
                        cval[out + r] = win[idx];
                    } else {
                        flag |= DERR_COUNT;
                    }
                    win[idx] = V(0);
                    r++;
                }
            }
            __syncthreads();
            written += wtot;
            __syncthreads();
        }
        if (written != expect) flag |= DERR_COUNT;
    }
    if (flag) atomicOr(err, flag);
}

// Cursor (8 B), next column (4 B) and long-row list slot (4 B) per stored
// entry of the longest row, for every resident block.
size_t window_global_ws(int64_t max_alen, int nsm) {
    return (size_t)(max_alen > 0 ? max_alen : 1) * 16 * (size_t)nsm * WIN_BPSM;
}

// ------------------------------------------------------------------ host side
template <typename K>
static int prep(K kern, size_t smem) {
    if (smem > 16 * 1024)
        SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return SPGEMM_OK;
}

static const char *NUM_LABEL[NBINS] = {"", "numeric.small", "numeric.small", "numeric.bin3",
                                       "numeric.bin4", "numeric.bin5", "numeric.bin6", ""};

template <int G, int MODE>
static int run_small(const NumP &a, const int4 *bdesc, int64_t n, const uint8_t *bins, DevState *st,
                     int *err, int maxbin, int slot_factor, Ctx &c) {
    constexpr int GPB = 256 / G;   // rows per block: 8 warps x 32/G rows
    const size_t smem = (size_t)GPB * SmallLayout<G>::stride * 4;
    SG_TRY(prep(k_num_small<G, MODE>, smem));
    int64_t blocks = (n + GPB - 1) / GPB;
    const int64_t cap = (int64_t)c.nsm * 32;
    blocks = blocks < cap ? blocks : cap;
    c.begin("numeric.small", n);
    k_num_small<G, MODE><<<(unsigned)blocks, 256, smem, c.s>>>(a, bdesc, n, bins, st, err, maxbin,
                                                                 slot_factor);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <int MODE>
static int run_small_g(const NumTune &t, const NumP &a, const int4 *bdesc, int64_t n, const uint8_t *bins,
                       DevState *st, int *err, Ctx &c) {
    const int maxbin = t.small_cap >= 32 ? 2 : 1;
    switch (t.G) {
        case 4: return run_small<4, MODE>(a, bdesc, n, bins, st, err, maxbin, t.slot_factor, c);
        case 8: return run_small<8, MODE>(a, bdesc, n, bins, st, err, maxbin, t.slot_factor, c);
        case 16: return run_small<16, MODE>(a, bdesc, n, bins, st, err, maxbin, t.slot_factor, c);
        default: return run_small<32, MODE>(a, bdesc, n, bins, st, err, maxbin, t.slot_factor, c);
    }
}

template <int BW, int NMAX, int WPB, int MODE>
static int run_rank(const NumP &a, const int4 *bdesc, const int2 *spans, const int32_t *rows, int64_t count,
                    int tier, DevState *st, int *err, const char *label, Ctx &c) {
    const size_t smem = RankLayout<BW, NMAX, WPB, MODE>::bytes;
    SG_TRY(prep(k_num_rank<BW, NMAX, WPB, MODE>, smem));
    int64_t blocks = (count + WPB - 1) / WPB;
    blocks = blocks < (int64_t)c.nsm * 32 ? blocks : (int64_t)c.nsm * 32;
    c.begin(label, count);
    k_num_rank<BW, NMAX, WPB, MODE><<<(unsigned)blocks, WPB * 32, smem, c.s>>>(a, bdesc, spans, rows, count,
                                                                                tier, st, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <int SMAX, int BW, int WPB, int MODE>
static int run_wide(const NumP &a, const int4 *bdesc, const int2 *spans, const int32_t *rows, int64_t count,
                    int min_nnz, int min_span, DevState *st, int *err, const char *label, Ctx &c) {
    const size_t smem = WideLayout<SMAX, BW, WPB, MODE>::bytes;
    SG_TRY(prep(k_num_wide<SMAX, BW, WPB, MODE>, smem));
    int64_t blocks = (count + WPB - 1) / WPB;
    blocks = blocks < (int64_t)c.nsm * 32 ? blocks : (int64_t)c.nsm * 32;
    c.begin(label, count);
    k_num_wide<SMAX, BW, WPB, MODE><<<(unsigned)blocks, WPB * 32, smem, c.s>>>(a, bdesc, spans, rows, count, min_nnz,
                                                                                min_span, st, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <int BS, int S, typename V>
static int run_block(const NumP &a, const int32_t *rows, int64_t count, int *err, int b, Ctx &c) {
    const size_t smem = (size_t)S * (sizeof(V) + 4) * 3 / 2 + (size_t)BLOCK_TAB * 16;
    SG_TRY(prep(k_num_block<BS, S, V>, smem));
    int64_t blocks = count < (int64_t)c.nsm * 16 ? count : (int64_t)c.nsm * 16;
    c.begin(NUM_LABEL[b], count);
    k_num_block<BS, S, V><<<(unsigned)blocks, BS, smem, c.s>>>(
        a.arp, a.acol, (const V *)a.aval, a.brp, a.bcol, (const V *)a.bval, a.crp, a.ccol,
        (V *)a.cval, rows, count, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

static int64_t huge_l2cap(int64_t max_row_nnz) {
    int64_t c = 2;
    while (c < 2 * max_row_nnz) c <<= 1;
    return c;
}

size_t numeric_global_ws(int64_t max_row_nnz, int64_t ncols_b, int nsm, int dtype) {
    const int64_t l2 = huge_l2cap(max_row_nnz);
    const int64_t nwords = (ncols_b + 31) / 32;
    const size_t vb = dtype == SPGEMM_F64 ? 8 : 4;
    return ((size_t)l2 * (4 + vb) + (size_t)nwords * 8) * (size_t)nsm;
}

template <typename V>
static int run_huge(const NumP &a, const spgemm_csr &B, const int32_t *rows, int64_t cnt, int *err,
                    void *gws, size_t gws_bytes, int64_t max_row_nnz, Ctx &c) {
    const int64_t l2 = huge_l2cap(max_row_nnz);
    const int64_t nwords = (B.ncols + 31) / 32;
    const int64_t blocks = cnt < (int64_t)c.nsm ? cnt : (int64_t)c.nsm;
    const size_t need = ((size_t)l2 * (4 + sizeof(V)) + (size_t)nwords * 8) * (size_t)blocks;
    if (need > gws_bytes) {
        set_error("numeric: global map workspace too small");
        return SPGEMM_ERR_INTERNAL;
    }
    const size_t smem = (size_t)HUGE_L1 * (sizeof(V) + 4);
    SG_TRY(prep(k_num_huge<V>, smem));
    c.begin("numeric.bin6", cnt);
    k_num_huge<V><<<(unsigned)blocks, HUGE_BS, smem, c.s>>>(
        a.arp, a.acol, (const V *)a.aval, a.brp, a.bcol, (const V *)a.bval, a.crp, a.ccol, (V *)a.cval,
        rows, cnt, err, l2, nwords, (unsigned char *)gws);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <typename V>
static int run_window(const NumP &a, const int32_t *rows, int64_t cnt, int *err, void *gws, size_t gws_bytes,
                      int64_t max_alen, Ctx &c) {
    constexpr int W = sizeof(V) == 8 ? 4096 : 8192;
    const int64_t cap = (int64_t)c.nsm * WIN_BPSM;
    const int64_t blocks = cnt < cap ? cnt : cap;
    if ((size_t)(max_alen > 0 ? max_alen : 1) * 16 * (size_t)blocks > gws_bytes) {
        set_error("numeric: cursor workspace too small");
        return SPGEMM_ERR_INTERNAL;
    }
    const size_t smem = (size_t)W * sizeof(V) + (size_t)(W / 32) * 4;
    SG_TRY(prep(k_num_window<V, W>, smem));
    c.begin("numeric.bin6_window", cnt);
    k_num_window<V, W><<<(unsigned)blocks, WIN_BS, smem, c.s>>>(
        a.arp, a.acol, (const V *)a.aval, a.brp, a.bcol, (const V *)a.bval, a.crp, a.ccol, (V *)a.cval, rows,
        cnt, err, max_alen, (unsigned char *)gws);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <int MODE>
static int run_all(const NumP &a, const spgemm_csr &A, const spgemm_csr &B, const uint8_t *bins,
                   const int4 *bdesc, const int2 *spans, const int32_t *rows, const long long *counts, DevState *st,
                   void *gws, size_t gws_bytes, int64_t max_row_nnz, const NumTune &t, bool b_sorted,
                   int64_t max_alen, Ctx &c) {
    using V = typename std::conditional<MODE == MODE_F32, float, double>::type;
    int *err = &st->err;
    const int first_list = t.small_cap >= 32 ? 3 : 2;
    if (counts[1] + (first_list == 3 ? counts[2] : 0) > 0)
        SG_TRY(run_small_g<MODE>(t, a, bdesc, A.nrows, bins, st, err, c));
    int64_t off = 0;
    for (int b = first_list; b <= BIN_HUGE; b++) {
        const int64_t cnt = counts[b];
        const int32_t *r = rows + off;
        const int2 *sp = spans + off;
        off += cnt;
        if (cnt == 0) continue;
        switch (b) {
            case 2:
            case 3:
            case 4:
                // dense rank accumulators for the rows rank_takes accepts (two span
                // limits), hash maps for the others (two map sizes)
                SG_TRY((run_rank<RANK_BW1, RANK_NMAX1, 8, MODE>(a, bdesc, sp, r, cnt, 1, st, err,
                                                                 "numeric.rank512", c)));
                SG_TRY((run_rank<RANK_BW2, RANK_NMAX2, 8, MODE>(a, bdesc, sp, r, cnt, 2, st, err,
                                                                 "numeric.rank1024", c)));
                SG_TRY((run_rank<RANK_BW3, RANK_NMAX3, 4, MODE>(a, bdesc, sp, r, cnt, 3, st, err,
                                                                 "numeric.rank2048", c)));
                // the rows left to the maps span more than RANK_BW3 words, so the
                // maps' own bitmap output (spans up to 32 * BW columns) is kept small
                if (b <= 3) {
                    SG_TRY((run_wide<256, 64, 8, MODE>(a, bdesc, sp, r, cnt, 0, 1, st, err, "numeric.wide3", c)));
                } else {
                    SG_TRY((run_wide<512, 64, 8, MODE>(a, bdesc, sp, r, cnt, 0, 1, st, err, "numeric.wide4a", c)));
                    SG_TRY((run_wide<1024, 64, 8, MODE>(a, bdesc, sp, r, cnt, 257, 1, st, err, "numeric.wide4b", c)));
                    SG_TRY((run_wide<2048, 64, 4, MODE>(a, bdesc, sp, r, cnt, 513, 1, st, err, "numeric.wide4c", c)));
                }
                break;
            case 5: SG_TRY((run_block<256, 8192, V>(a, r, cnt, err, b, c))); break;
            default:
                if (b_sorted) SG_TRY(run_window<V>(a, r, cnt, err, gws, gws_bytes, max_alen, c));
                else SG_TRY(run_huge<V>(a, B, r, cnt, err, gws, gws_bytes, max_row_nnz, c));
        }
    }
    return SPGEMM_OK;
}

int launch_numeric(int dtype, bool f64_native, const spgemm_csr &A, const spgemm_csr &B, spgemm_csr &C,
                   const uint8_t *bins, const int4 *bdesc, const int2 *spans, const int32_t *rows,
                   const long long *counts, DevState *st, float2 *bsplit, void *gws,
                   size_t gws_bytes, int64_t max_row_nnz, const NumTune &G, bool b_sorted,
                   int64_t max_alen, Ctx &c) {
    NumP a{A.row_ptr, A.col_idx, A.values, B.row_ptr, B.col_idx, B.values, bsplit,
           C.row_ptr, C.col_idx, C.values};
    if (dtype == SPGEMM_F32)
        return run_all<MODE_F32>(a, A, B, bins, bdesc, spans, rows, counts, st, gws, gws_bytes, max_row_nnz, G, b_sorted, max_alen, c);
    if (f64_native)
        return run_all<MODE_F64>(a, A, B, bins, bdesc, spans, rows, counts, st, gws, gws_bytes, max_row_nnz, G, b_sorted, max_alen, c);
    SG_CUDA(cudaMemsetAsync(&st->b_out_of_range, 0, sizeof(int), c.s));
    if (B.nnz > 0) {
        int64_t blocks = (B.nnz + 255) / 256;
        blocks = blocks < (int64_t)c.nsm * 16 ? blocks : (int64_t)c.nsm * 16;
        c.begin("numeric.split_b", B.nnz);
        k_split_values<<<(unsigned)blocks, 256, 0, c.s>>>(B.nnz, (const double *)B.values, bsplit, st);
        c.end();
        SG_CUDA(cudaGetLastError());
    }
    return run_all<MODE_DW>(a, A, B, bins, bdesc, spans, rows, counts, st, gws, gws_bytes, max_row_nnz, G, b_sorted, max_alen, c);
}

}  // namespace sg
