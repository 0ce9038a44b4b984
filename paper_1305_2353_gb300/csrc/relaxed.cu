// relaxed.cu -- K2: relaxed compression of A21 (Section 4.2).
//
// The paper's construction is sequential: for j = 1..p, the unflagged row with
// the largest |a21(i,j)| (lowest row on ties) is flagged and copied into row j
// of C.  Before column j at most j-1 rows are flagged, so its choice is always
// among the K_j = j+1 largest entries of column j in the order (|a| desc, row
// asc).  The GPU form is exact and reads A21 once:
//   pass 1  (HBM-bound) block maxima: for every column and every block of B
//           consecutive rows (B = 64 when there are enough rows), the largest
//           key of the block;
//   pass 2  one CTA per column: thr = the K_j-th largest block maximum.  The
//           K_j blocks with maxima >= thr hold K_j distinct entries >= thr, so
//           the K_j-th largest entry of the column is >= thr, and every entry
//           of the top K_j lies in a block whose maximum is >= thr.  Those
//           blocks are read again (about K_j * B rows, from L2 or HBM), their
//           entries >= thr collected and sorted, and the first K_j kept;
//   pass 3  one CTA runs the paper's greedy over the sorted lists, a warp
//           testing a column's leading candidates at once;
//   pass 4  the chosen rows are gathered, with their signs, into C.
// Where ties leave more candidates than shared memory holds, pass 2 streams
// the whole column instead (the top-K of a running threshold, below), which is
// also how one row block of a row-split supernode builds its lists.
// Magnitudes are compared as integer keys (sign bit cleared), so no FP64
// arithmetic is involved and the result is bit-exact.
#include "ctp_internal.cuh"
#include "tc_common.cuh"

namespace ctp {

namespace {

constexpr int kT1 = 512;      // threads per CTA of the column kernels
constexpr int kCap = 4096;    // candidate buffer (power of two)
constexpr int kChunk = 2048;  // rows read per pass (4 per thread)
constexpr unsigned long long kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long kInfKey = 0x7FF0000000000000ull;

struct Cand {
    unsigned long long key;  // |a| as an integer key
    int row;                 // A21 row
    int pad;
};

// a precedes b in the paper's order: larger magnitude first, lower row on ties
__device__ __forceinline__ bool before(const Cand &a, const Cand &b) {
    return a.key > b.key || (a.key == b.key && a.row < b.row);
}

// Sort (key, row)[0..N) (N a power of two) into the paper's order (larger
// magnitude first, lower row on ties).  Keys and rows live in separate arrays
// so that each thread's accesses are 8- and 4-byte words (few bank conflicts).
__device__ void bitonic_desc(unsigned long long *key, int *row, int N) {
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
                // t-th pair of this phase: i has bit j clear
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const int ixj = i | j;
                const unsigned long long ka = key[i], kb = key[ixj];
                const int ra = row[i], rb = row[ixj];
                const bool a_first = ka > kb || (ka == kb && ra < rb);
                const bool first_block = (i & k) == 0;  // this block descends
                if (first_block != a_first) {
                    key[i] = kb;
                    key[ixj] = ka;
                    row[i] = rb;
                    row[ixj] = ra;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int next_pow2(int x) {
    int n = 1;
    while (n < x) n <<= 1;
    return n;
}

// The K-th largest of the keys a CTA holds (keys with the top bit clear),
// found digit by digit (8 bits at a time) with a 256-bin histogram in shared
// memory: exact, and no sort.  Every thread passes its keys through `each(f)`:
// f(key, valid) is called by all 32 lanes of a warp together (valid = false
// for a lane without a key in that call), so that lanes with the same digit
// add to their bin with one atomic (close keys share their leading digits).
struct RadixScratch {
    unsigned hist[256];
    unsigned long long prefix;
    int k;
};
template <typename Each>
__device__ unsigned long long kth_largest(int K, RadixScratch &rs, Each each) {
    unsigned long long prefix = 0, mask = 0;
    int k = K;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) rs.hist[b] = 0;
        __syncthreads();
        each([&](unsigned long long v, bool valid) {
            const bool in = valid && (v & mask) == prefix;
            const unsigned bin = in ? (unsigned)((v >> shift) & 255u) : 256u;
            const unsigned grp = __match_any_sync(0xffffffffu, bin);
            if (in && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&rs.hist[bin], (unsigned)__popc(grp));
        });
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane l sums bins 255-8l .. 248-8l (descending order of digits)
            const int lane = threadIdx.x;
            unsigned cnt[8], tot = 0;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                cnt[q] = rs.hist[255 - 8 * lane - q];
                tot += cnt[q];
            }
            unsigned incl = tot;  // inclusive prefix over lanes (larger digits first)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned excl = incl - tot;
            // the lane whose range holds the k-th largest
            if (excl < (unsigned)k && (unsigned)k <= incl) {
                unsigned c = excl;
                int d = 255 - 8 * lane;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    if (c + cnt[q] >= (unsigned)k) {
                        d = 255 - 8 * lane - q;
                        break;
                    }
                    c += cnt[q];
                }
                rs.prefix = prefix | ((unsigned long long)d << shift);
                rs.k = k - (int)c;
            }
        }
        __syncthreads();
        prefix = rs.prefix;
        k = rs.k;
        mask |= 0xFFull << shift;
        __syncthreads();
    }
    return prefix;
}

// Append the (key, row) pairs with keep = true to the buffer, one shared atomic
// per warp (the order inside the buffer does not matter).
__device__ __forceinline__ void warp_append(bool keep, unsigned long long kv, int rw, unsigned long long *key,
                                            int *row, int *cnt) {
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (bal == 0) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(bal) - 1) base = atomicAdd(cnt, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
    if (keep) {
        const int at = base + __popc(bal & ((1u << lane) - 1u));
        key[at] = kv;
        row[at] = rw;
    }
}

// Keep the buffer entries with key >= thr, in place (every thread reads its
// entries before the barrier and writes after it).
__device__ void compact_ge(unsigned long long thr, unsigned long long *key, int *row, int *cnt, int *wsum) {
    const int n = *cnt;
    constexpr int kPerT = kCap / kT1;
    unsigned long long kk[kPerT];
    int rr[kPerT];
    bool kp[kPerT];
    int mine = 0;
#pragma unroll
    for (int q = 0; q < kPerT; q++) {
        const int i = threadIdx.x * kPerT + q;  // contiguous runs keep the order stable
        kp[q] = i < n && key[i] >= thr;
        kk[q] = i < n ? key[i] : 0;
        rr[q] = i < n ? row[i] : 0;
        mine += kp[q] ? 1 : 0;
    }
    // exclusive scan of `mine` over the CTA
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < kT1 / 32 ? wsum[threadIdx.x] : 0, in2 = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, in2, o);
            if (threadIdx.x >= o) in2 += y;
        }
        if (threadIdx.x < kT1 / 32) wsum[threadIdx.x] = in2 - v;  // exclusive, per warp
        if (threadIdx.x == kT1 / 32 - 1) wsum[kT1 / 32] = in2;    // total
    }
    __syncthreads();
    int at = wsum[w] + incl - mine;
#pragma unroll
    for (int q = 0; q < kPerT; q++)
        if (kp[q]) {
            key[at] = kk[q];
            row[at] = rr[q];
            ++at;
        }
    __syncthreads();
    if (threadIdx.x == 0) *cnt = wsum[kT1 / 32];
    __syncthreads();
}

// The top K entries of rows [r0, r1) of one column, streamed: each pass reads
// kChunk rows, four per thread, with the next chunk's loads in flight.  A
// threshold thr (a lower bound of the K-th largest key of the rows, taken as
// the K-th largest of what was seen so far by radix selection) filters the
// stream, so only entries >= thr reach the shared buffer (ties kept: a
// superset of the top K); when the buffer fills, the threshold is raised and
// the buffer filtered again.  On return the buffer key/row[0..cnt) holds the
// top K plus ties, sorted into the paper's order (|a| descending, lower row
// first), cnt >= min(K, r1 - r0).  Rows are reported relative to the column.
__device__ void stream_topk(const double *__restrict__ col, int64_t r0, int64_t r1, int K,
                            unsigned long long *key, int *row, int &cnt, int *wsum, RadixScratch &rs,
                            bool &nonfinite) {
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    bool have_thr = false;
    // thr: the K-th largest key among the rows seen so far.  A later row whose
    // key equals it ranks after every earlier tie (rows only grow along the
    // stream), so it cannot enter the top K: later rows need key > thr.
    unsigned long long thr = 0;
    auto buffer_each = [&](auto f) {
        for (int i0 = 0; i0 < cnt; i0 += kT1) {
            const int i = i0 + threadIdx.x;
            f(i < cnt ? key[i] : 0ull, i < cnt);
        }
    };
    constexpr int kPer = kChunk / kT1;
    double vn[kPer];
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        const int64_t r = r0 + q * kT1 + threadIdx.x;
        vn[q] = (r < r1) ? __ldcs(col + r) : 0.0;
    }
    for (int64_t base = r0; base < r1; base += kChunk) {
        double v[kPer];
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            v[q] = vn[q];
            const int64_t r = base + kChunk + q * kT1 + threadIdx.x;
            vn[q] = (r < r1) ? __ldcs(col + r) : 0.0;
        }
        unsigned long long kv[kPer];
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const int64_t r = base + q * kT1 + threadIdx.x;
            kv[q] = (unsigned long long)__double_as_longlong(v[q]) & kAbsMask;
            nonfinite |= (r < r1) && kv[q] >= kInfKey;
        }
        const int64_t nin = (r1 - base) < kChunk ? (r1 - base) : kChunk;
        bool fresh = false;  // thr taken from this chunk: its own ties stay
        if (!have_thr && cnt == 0 && nin >= K && K > 0) {
            // the first chunk alone holds K entries: its K-th largest is a valid threshold
            thr = kth_largest(K, rs, [&](auto f) {
#pragma unroll
                for (int q = 0; q < kPer; q++) f(kv[q], base + q * kT1 + threadIdx.x < r1);
            });
            have_thr = true;
            fresh = true;
        }
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const int64_t r = base + q * kT1 + threadIdx.x;
            const bool keep = r < r1 && (!have_thr || kv[q] > thr || (fresh && kv[q] == thr));
            warp_append(keep, kv[q], (int)(r - r0), key, row, &cnt);
        }
        __syncthreads();
        // room for another chunk: raise the threshold and filter when needed
        if (cnt > kCap - kChunk || (!have_thr && cnt >= K && K > 0)) {
            thr = kth_largest(K, rs, buffer_each);
            have_thr = true;
            compact_ge(thr, key, row, &cnt, wsum);
            if (cnt > kCap - kChunk) {
                // many entries tie with the threshold: sort and keep exactly the
                // first K
                const int N = next_pow2(cnt);
                for (int i = cnt + threadIdx.x; i < N; i += kT1) {
                    key[i] = 0;
                    row[i] = 0x7fffffff;
                }
                __syncthreads();
                bitonic_desc(key, row, N);
                thr = key[K - 1];
                __syncthreads();
                if (threadIdx.x == 0) cnt = K;
                __syncthreads();
            }
        }
    }
    // survivors: the top K plus ties, sorted once
    if (have_thr && cnt > K) {
        const unsigned long long t2 = kth_largest(K, rs, buffer_each);
        compact_ge(t2, key, row, &cnt, wsum);
    }
    const int n = cnt, N = next_pow2(n > 1 ? n : 1);
    for (int i = n + threadIdx.x; i < N; i += kT1) {
        key[i] = 0;
        row[i] = 0x7fffffff;  // padding sorts last
    }
    __syncthreads();
    bitonic_desc(key, row, N);
}

// Write the first k of the sorted buffer as list `slot` of column j.
__device__ void write_list(const unsigned long long *key, const int *row, int n, int K, int j, int nslot, int slot,
                           int row0, int p, Cand *__restrict__ lists, int *__restrict__ lens) {
    const int k = n < K ? n : K;
    const int li = j * nslot + slot;
    Cand *out = lists + (int64_t)li * p;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        Cand c;
        c.key = key[i];
        c.row = row0 + row[i];
        c.pad = 0;
        out[i] = c;
    }
    if (threadIdx.x == 0) lens[li] = k;
}

// One row block of A21 (a row-split supernode, Section 6): CTA j streams
// column j and writes its top K_j as list `slot` of nslot.
__global__ void __launch_bounds__(kT1)
    k_relaxed_topk(const double *__restrict__ A21, int64_t m, int p, int64_t lda, int slot, int nslot, int row0,
                   Cand *__restrict__ lists, int *__restrict__ lens, int32_t *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *key = reinterpret_cast<unsigned long long *>(smraw);  // [kCap]
    int *row = reinterpret_cast<int *>(key + kCap);                           // [kCap]
    __shared__ int cnt;
    __shared__ int wsum[kT1 / 32 + 1];
    __shared__ RadixScratch rs;
    const int j = blockIdx.x;
    const int K = (int)((int64_t)j + 1 < m ? (int64_t)j + 1 : m);
    bool nonfinite = false;
    stream_topk(A21 + (int64_t)j * lda, 0, m, K, key, row, cnt, wsum, rs, nonfinite);
    write_list(key, row, cnt, K, j, nslot, slot, row0, p, lists, lens);
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
}

// Pass 1: bmax[j * nb + b] = the largest key of rows [b*B, (b+1)*B) of column
// j (B = 2^lgB <= 64; rows past m count as 0).  A warp reads 64 consecutive
// rows of one column per load (two per lane, 16 bytes when A21 allows), four
// such pieces (2 KB in a row) in flight.  The pieces are numbered down the
// columns and dealt to the warps in groups of four, round robin, so that the
// warps of the whole grid sweep A21 together from one end to the other (the
// open DRAM pages stay few).  kFull: B = 64, the warp's maximum by two
// reductions of the 32-bit halves of the keys.
template <bool kVec, bool kFull>
__global__ void __launch_bounds__(256)
    k_block_max(const double *__restrict__ A21, int64_t m, int p, int64_t lda, int lgB, int64_t nb,
                unsigned long long *__restrict__ bmax, int32_t *__restrict__ info) {
    constexpr int kU = 4;
    const int lane = threadIdx.x & 31;
    const int nc = (int)((m + 63) >> 6);  // 64-row pieces per column
    const int gw = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    // piece u = j * nc + c: this warp starts at u = kU * gw and steps by kU * nw
    const int64_t step = (int64_t)kU * nw;
    const int sj = (int)(step / nc), sc = (int)(step - (int64_t)sj * nc);
    int j = (int)(((int64_t)kU * gw) / nc), c = (int)((int64_t)kU * gw - (int64_t)j * nc);
    bool nonfinite = false;
    while (j < p) {
        unsigned long long x0[kU], x1[kU];
        int jq[kU], cq[kU];
        int jj = j, cc = c;
#pragma unroll
        for (int q = 0; q < kU; q++) {
            jq[q] = jj;
            cq[q] = cc;
            x0[q] = x1[q] = 0;
            if (jj < p) {
                const int64_t r = ((int64_t)cc << 6) + 2 * lane;
                const double *a = A21 + (int64_t)jj * lda + r;
                if (kVec && r + 1 < m) {
                    const double2 v = __ldcs(reinterpret_cast<const double2 *>(a));
                    x0[q] = (unsigned long long)__double_as_longlong(v.x);
                    x1[q] = (unsigned long long)__double_as_longlong(v.y);
                } else {
                    if (r < m) x0[q] = (unsigned long long)__double_as_longlong(__ldcs(a));
                    if (r + 1 < m) x1[q] = (unsigned long long)__double_as_longlong(__ldcs(a + 1));
                }
            }
            if (++cc == nc) {
                cc = 0;
                ++jj;
            }
        }
#pragma unroll
        for (int q = 0; q < kU; q++) {
            if (jq[q] >= p) break;  // warp-uniform
            const unsigned long long a0 = x0[q] & kAbsMask, a1 = x1[q] & kAbsMask;
            unsigned long long *out = bmax + (int64_t)jq[q] * nb;
            if (kFull) {
                const unsigned long long v = a0 > a1 ? a0 : a1;
                const unsigned h = (unsigned)(v >> 32);
                const unsigned H = __reduce_max_sync(0xffffffffu, h);
                const unsigned L = __reduce_max_sync(0xffffffffu, h == H ? (unsigned)v : 0u);
                nonfinite |= H >= 0x7FF00000u;
                if (lane == q) out[cq[q]] = ((unsigned long long)H << 32) | L;
                continue;
            }
            if (lgB == 0) {
                const int64_t b = ((int64_t)cq[q] << 6) + 2 * lane;
                nonfinite |= a0 >= kInfKey || a1 >= kInfKey;
                if (b < nb) out[b] = a0;
                if (b + 1 < nb) out[b + 1] = a1;
                continue;
            }
            unsigned long long v = a0 > a1 ? a0 : a1;
            for (int o = 1; o < (1 << (lgB - 1)); o <<= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
                v = w > v ? w : v;
            }
            nonfinite |= v >= kInfKey;
            const int64_t b = ((int64_t)cq[q] << (6 - lgB)) + (lane >> (lgB - 1));  // B/2 lanes per block
            if ((lane & ((1 << (lgB - 1)) - 1)) == 0 && b < nb) out[b] = v;
        }
        j += sj;
        c += sc;
        if (c >= nc) {
            c -= nc;
            j++;
        }
    }
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
}

// Pass 1 with the tiles brought in by TMA (64-row pieces of 32 columns, 16 KB,
// six in flight per CTA, two CTAs per SM): the copies keep some 200 KB per SM
// on the way from HBM without holding registers, which is what a stream at
// full HBM speed needs (the per-warp loads above hold too few bytes in flight).
// Warp w of 8 reduces columns w, w + 8, w + 16, w + 24 of each tile (each
// column's 64 rows are 512 contiguous bytes of the tile); a ninth warp issues
// the copies.  Every wait is bounded.
constexpr int kBmR = 64, kBmC = 32;  // tile: rows x columns
constexpr int kBmStages = 6;
constexpr int kBmWarps = 8;
constexpr int kBmThreads = 32 * (kBmWarps + 1);
__global__ void __launch_bounds__(kBmThreads, 2)
    k_block_max_tma(const __grid_constant__ CUtensorMap map, int64_t m, int p, int64_t nb,
                    unsigned long long *__restrict__ bmax, int32_t *__restrict__ info) {
    extern __shared__ unsigned char smraw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ unsigned long long full[kBmStages], empty[kBmStages];
    __shared__ int abort_flag;
    constexpr uint32_t kTileBytes = kBmR * kBmC * 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nc = (int)((m + kBmR - 1) / kBmR), ng = (p + kBmC - 1) / kBmC;
    const int64_t ntiles = (int64_t)nc * ng;
    const int64_t nk = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kBmStages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kBmWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == kBmWarps) {
        // ---- producer: tile k of this CTA into stage k mod S once tile k - S is released
        if (lane == 0) {
            int64_t issued = 0;
            bool ok = true;
            for (int64_t k = 0; k < nk; k++) {
                const int s = (int)(k % kBmStages);
                if (k >= kBmStages &&
                    !tc::mbar_wait(&empty[s], (uint32_t)((k / kBmStages - 1) & 1), &abort_flag)) {
                    ok = false;
                    break;
                }
                const int64_t t = blockIdx.x + k * gridDim.x;
                const int g = (int)(t / nc), c = (int)(t - (int64_t)g * nc);
                tc::mbar_expect_tx(&full[s], kTileBytes);
                tc::tma_load_2d(tiles + (size_t)s * kTileBytes, &map, c * kBmR, g * kBmC, &full[s]);
                issued = k + 1;
            }
            if (!ok) {
                atomicExch(&abort_flag, 1);
                atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
                int never = 0;  // the shared memory must outlive the copies into it
                for (int64_t k = issued > kBmStages ? issued - kBmStages : 0; k < issued; k++)
                    tc::mbar_wait(&full[k % kBmStages], (uint32_t)((k / kBmStages) & 1), &never);
            }
        }
        return;
    }
    bool nonfinite = false;
    for (int64_t k = 0; k < nk; k++) {
        const int s = (int)(k % kBmStages);
        if (!tc::mbar_wait(&full[s], (uint32_t)((k / kBmStages) & 1), &abort_flag)) {
            if (lane == 0) {
                atomicExch(&abort_flag, 1);
                atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
            }
            break;
        }
        const uint8_t *tile = tiles + (size_t)s * kTileBytes;
        unsigned long long v[kBmC / kBmWarps];
#pragma unroll
        for (int q = 0; q < kBmC / kBmWarps; q++) {
            const ulonglong2 x =
                *reinterpret_cast<const ulonglong2 *>(tile + (warp + q * kBmWarps) * (kBmR * 8) + lane * 16);
            const unsigned long long a0 = x.x & kAbsMask, a1 = x.y & kAbsMask;
            v[q] = a0 > a1 ? a0 : a1;
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[s]);  // the tile is in registers
        const int64_t t = blockIdx.x + k * gridDim.x;
        const int g = (int)(t / nc), c = (int)(t - (int64_t)g * nc);
#pragma unroll
        for (int q = 0; q < kBmC / kBmWarps; q++) {
            const int j = g * kBmC + warp + q * kBmWarps;
            const unsigned h = (unsigned)(v[q] >> 32);
            const unsigned H = __reduce_max_sync(0xffffffffu, h);
            const unsigned L = __reduce_max_sync(0xffffffffu, h == H ? (unsigned)v[q] : 0u);
            if (j < p) {
                nonfinite |= H >= 0x7FF00000u;
                if (lane == q) bmax[(int64_t)j * nb + c] = ((unsigned long long)H << 32) | L;
            }
        }
    }
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
}

constexpr int kCblk = 2048;  // candidate blocks a column may have in pass 2

// Pass 2: CTA j finds the top K_j of column j from the block maxima (see the
// top of the file) and writes it as list `slot` of nslot.
__global__ void __launch_bounds__(kT1)
    k_relaxed_pick(const double *__restrict__ A21, int64_t m, int p, int64_t lda, int lgB, int64_t nb,
                   const unsigned long long *__restrict__ bmax, int slot, int nslot, int row0,
                   Cand *__restrict__ lists, int *__restrict__ lens, int32_t *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *key = reinterpret_cast<unsigned long long *>(smraw);  // [kCap]
    int *row = reinterpret_cast<int *>(key + kCap);                           // [kCap]
    __shared__ int cblk[kCblk];
    __shared__ int cnt, ncb;
    __shared__ int wsum[kT1 / 32 + 1];
    __shared__ RadixScratch rs;
    const int j = blockIdx.x;
    const int K = (int)((int64_t)j + 1 < m ? (int64_t)j + 1 : m);
    const double *col = A21 + (int64_t)j * lda;
    const unsigned long long *bm = bmax + (int64_t)j * nb;
    const int B = 1 << lgB;
    if (threadIdx.x == 0) {
        cnt = 0;
        ncb = 0;
    }
    // (a) thr = the K-th largest block maximum (nb >= K by the choice of B)
    const bool cached = nb <= kCap;
    if (cached)
        for (int i = threadIdx.x; i < nb; i += kT1) key[i] = __ldcg(bm + i);
    __syncthreads();
    const unsigned long long thr = kth_largest(K, rs, [&](auto f) {
        for (int64_t i0 = 0; i0 < nb; i0 += kT1) {
            const int64_t i = i0 + threadIdx.x;
            f(i < nb ? (cached ? key[i] : __ldcg(bm + i)) : 0ull, i < nb);
        }
    });
    // (b) the blocks whose maximum reaches thr
    for (int64_t i0 = 0; i0 < nb; i0 += kT1) {
        const int64_t i = i0 + threadIdx.x;
        const bool in = i < nb && (cached ? key[i] : __ldcg(bm + i)) >= thr;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (bal == 0) continue;
        int base = 0;
        const int lane = threadIdx.x & 31;
        if (lane == __ffs(bal) - 1) base = atomicAdd(&ncb, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
        const int at = base + __popc(bal & ((1u << lane) - 1u));
        if (in && at < kCblk) cblk[at] = (int)i;
    }
    __syncthreads();  // the cached maxima are no longer needed: key/row take candidates
    const int nblk = ncb;
    bool overflow = nblk > kCblk;
    if (!overflow) {
        // (c) their entries >= thr (a superset of the top K), four loads in flight per thread
        const int64_t total = (int64_t)nblk << lgB;
        for (int64_t f0 = 0; f0 < total; f0 += 4 * kT1) {
            unsigned long long kv[4];
            int64_t rr[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int64_t f = f0 + q * kT1 + threadIdx.x;
                rr[q] = -1;
                kv[q] = 0;
                if (f < total) {
                    const int64_t r = ((int64_t)cblk[f >> lgB] << lgB) + (f & (B - 1));
                    if (r < m) {
                        rr[q] = r;
                        kv[q] = (unsigned long long)__double_as_longlong(__ldcg(col + r)) & kAbsMask;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const bool keep = rr[q] >= 0 && kv[q] >= thr;
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (bal == 0) continue;
                const int lane = threadIdx.x & 31;
                int base = 0;
                if (lane == __ffs(bal) - 1) base = atomicAdd(&cnt, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
                const int at = base + __popc(bal & ((1u << lane) - 1u));
                if (keep && at < kCap) {
                    key[at] = kv[q];
                    row[at] = (int)rr[q];
                }
            }
        }
        // (every thread decides before the streaming path may reset cnt)
        overflow = __syncthreads_or(cnt > kCap);
    }
    bool nonfinite = false;
    if (overflow) {
        // many ties: stream the column
        stream_topk(col, 0, m, K, key, row, cnt, wsum, rs, nonfinite);
    } else {
        const int n = cnt, N = next_pow2(n > 1 ? n : 1);
        for (int i = n + threadIdx.x; i < N; i += kT1) {
            key[i] = 0;
            row[i] = 0x7fffffff;  // padding sorts last
        }
        __syncthreads();
        bitonic_desc(key, row, N);
    }
    write_list(key, row, cnt, K, j, nslot, slot, row0, p, lists, lens);
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
}

// Pass 3: the greedy of Section 4.2 over the candidate lists (nseg sorted
// lists per column), then optionally the gather of the chosen rows into C.
//   (a) the first hd entries of every list (hd = 32 / nseg, at least 4) are
//       copied into shared memory by all threads at once; then thread j merges
//       column j's runs into one sorted prefix, exact up to the smallest
//       staged entry of any list that holds more;
//   (b) one warp runs the sequential greedy: for column j its lanes test the
//       entries of the exact prefix against the chosen rows at once (a bitmap
//       over the rows when they fit in shared memory, else a small
//       open-addressing hash set) and the first free entry is taken; a column
//       whose exact prefix is all taken falls back to walking the full lists
//       in global memory.
constexpr int kHash = 1024;                  // > 2 * kMaxP slots
constexpr int64_t kBitmapRows = 64 * 8192;   // rows a 64 KB bitmap covers

__host__ __device__ inline int greedy_head(int nseg) {
    const int h = 32 / nseg;
    return h < 4 ? 4 : h;
}

__device__ __forceinline__ unsigned hslot(int row) { return ((unsigned)row * 2654435761u) >> 22; }
__device__ __forceinline__ bool hash_has(const int *set, int row) {
    for (unsigned h = hslot(row) & (kHash - 1);; h = (h + 1) & (kHash - 1)) {
        if (set[h] == row) return true;
        if (set[h] < 0) return false;
    }
}
__device__ __forceinline__ void hash_put(int *set, int row) {
    unsigned h = hslot(row) & (kHash - 1);
    while (set[h] >= 0) h = (h + 1) & (kHash - 1);
    set[h] = row;
}

// Slow path of the greedy for column j: walk its nseg sorted lists in global
// memory in merged order and return the first row not chosen yet (-1: none).
__device__ __noinline__ int greedy_walk(int j, int nseg, int p, const Cand *__restrict__ lists,
                                        const int *__restrict__ lens, bool use_bits, const unsigned *bits,
                                        const int *hset) {
    int head[8];
    for (int s = 0; s < nseg; s++) head[s] = 0;
    for (;;) {
        int bs = -1;
        Cand best;
        best.key = 0;
        best.row = 0x7fffffff;
        for (int s = 0; s < nseg; s++) {
            const int li = j * nseg + s;
            if (head[s] < lens[li]) {
                const Cand c = lists[(int64_t)li * p + head[s]];
                if (bs < 0 || before(c, best)) {
                    best = c;
                    bs = s;
                }
            }
        }
        if (bs < 0) return -1;
        const int rb = best.row;
        if (!(use_bits ? ((bits[rb >> 5] >> (rb & 31)) & 1u) != 0 : hash_has(hset, rb))) return rb;
        head[bs]++;
    }
}

// rmax > 0: every candidate row is below rmax <= kBitmapRows (the bitmap is used)
constexpr int kGreedyThreads = 512;
__global__ void __launch_bounds__(kGreedyThreads)
    k_relaxed_greedy(const double *__restrict__ A21, int64_t lda, int p, int nseg,
                     const Cand *__restrict__ lists, const int *__restrict__ lens,
                     double *__restrict__ C, int32_t *__restrict__ rows_out, int rmax) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int hd = greedy_head(nseg);
    const int W = nseg * hd;                                         // merged prefix width (<= 32)
    // entry e of column j at mrg[e * p + j]: the threads (lanes) of consecutive
    // columns touch consecutive entries (no bank conflicts)
    Cand *mrg = reinterpret_cast<Cand *>(gsm);                       // [W][p]
    int *mlen = reinterpret_cast<int *>(mrg + (size_t)p * W);        // [p] exact prefix length
    unsigned *bits = reinterpret_cast<unsigned *>(mlen + p);         // [rmax / 32] chosen rows
    __shared__ int chosen[kMaxP];
    __shared__ int hset[kHash];
    const bool use_bits = rmax > 0;
    for (int i = threadIdx.x; i < kHash; i += blockDim.x) hset[i] = -1;
    if (use_bits)
        for (int i = threadIdx.x; i < (rmax + 31) / 32; i += blockDim.x) bits[i] = 0u;
    // (a) staged heads: list (j, s) entry q at position s*hd + q of column j,
    // eight loads in flight per thread (an entry is read before its list's
    // length is known and kept only when it exists)
    const int nstage = p * W;
    constexpr int kSU = 8;
    for (int base = 0; base < nstage; base += kSU * blockDim.x) {
        Cand v[kSU];
        bool ok[kSU];
#pragma unroll
        for (int u = 0; u < kSU; u++) {
            const int idx = base + u * blockDim.x + threadIdx.x;
            const int li = idx / hd, q = idx - li * hd;  // li = j * nseg + s
            ok[u] = idx < nstage && q < p;
            if (ok[u]) v[u] = lists[(int64_t)li * p + q];
            ok[u] = ok[u] && q < lens[li];
        }
#pragma unroll
        for (int u = 0; u < kSU; u++)
            if (ok[u]) {
                const int idx = base + u * blockDim.x + threadIdx.x;
                const int j = idx / W;
                mrg[(size_t)(idx - j * W) * p + j] = v[u];
            }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        if (nseg == 1) {  // one sorted list: its staged head is the exact prefix
            const int len = lens[j];
            mlen[j] = len < hd ? len : hd;
            continue;
        }
        Cand *out = mrg + j;  // entry e at out[e * p]
        int cnt = 0;
        bool have_lim = false;
        Cand lim;
        lim.key = 0;
        lim.row = 0x7fffffff;
        for (int s = 0; s < nseg; s++) {
            const int len = lens[j * nseg + s];
            const int h = len < hd ? len : hd;
            if (len > hd) {
                // entries beyond this list's staged ones may come after its last staged entry
                const Cand last = out[(size_t)(s * hd + hd - 1) * p];
                if (!have_lim || before(last, lim)) {
                    lim = last;
                    have_lim = true;
                }
            }
            for (int q = 0; q < h; q++) {  // insertion into the sorted prefix out[0..cnt)
                const Cand c = out[(size_t)(s * hd + q) * p];
                int at = cnt++;
                while (at > 0 && before(c, out[(size_t)(at - 1) * p])) {
                    out[(size_t)at * p] = out[(size_t)(at - 1) * p];
                    --at;
                }
                out[(size_t)at * p] = c;
            }
        }
        int exact = cnt;
        if (have_lim) {
            exact = 0;
            while (exact < cnt && !before(lim, out[(size_t)exact * p])) ++exact;  // out[exact] <= lim in order
        }
        mlen[j] = exact;
    }
    __syncthreads();
    // (b) the greedy, one warp
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        auto walk = [&](int j) { return greedy_walk(j, nseg, p, lists, lens, use_bits, bits, hset); };
        if (use_bits) {
            // 32 columns at a time, lane l taking column j0 + l.  Columns j0..F-1
            // are settled; every other lane proposes the first entry of its exact
            // prefix that is not chosen yet.  Column k's sequential choice is its
            // proposal unless a lower unsettled lane proposes the same row (its
            // earlier entries are all chosen rows already), so the lanes from F
            // up to the first repeated proposal settle together, and the rest
            // propose again.  A lane that runs out of exact entries settles
            // alone, by the slow path, once it is the lowest unsettled lane.
            for (int j0 = 0; j0 < p; j0 += 32) {
                const int j = j0 + lane;
                const int nl = p - j0 < 32 ? p - j0 : 32;
                const Cand *pre = mrg + (j < p ? j : 0);  // entry e at pre[e * p]
                const int ex = j < p ? mlen[j] : 0;
                int pos = 0;
                int F = 0;
                while (F < nl) {
                    int r = -2;  // -2: needs the slow path
                    if (lane >= F && lane < nl) {
                        int rp = pos < ex ? pre[(size_t)pos * p].row : -1;
                        while (rp >= 0 && ((bits[rp >> 5] >> (rp & 31)) & 1u)) {
                            pos++;
                            rp = pos < ex ? pre[(size_t)pos * p].row : -1;
                        }
                        if (rp >= 0) r = rp;
                    }
                    const unsigned slow = __ballot_sync(0xffffffffu, lane >= F && lane < nl && r == -2);
                    // the first repeated proposal among the unsettled lanes
                    const unsigned same = __match_any_sync(0xffffffffu, (lane >= F && lane < nl && r >= 0) ? r : -3 - lane);
                    const unsigned below = (1u << lane) - 1u;
                    const bool dup = lane >= F && lane < nl && r >= 0 && (same & below & ~((1u << F) - 1u)) != 0;
                    unsigned stop = __ballot_sync(0xffffffffu, dup) | slow;
                    int L = stop ? __ffs(stop) - 1 : nl;
                    if (L > nl) L = nl;
                    if (L == F) {
                        // lane F needs the slow path: every lower column is settled
                        int rs = -1;
                        if (lane == F) rs = walk(j);
                        rs = __shfl_sync(0xffffffffu, rs, F);
                        if (lane == F) {
                            chosen[j] = rs;
                            if (rs >= 0) atomicOr(&bits[rs >> 5], 1u << (rs & 31));
                        }
                        L = F + 1;
                    } else if (lane >= F && lane < L) {
                        chosen[j] = r;
                        atomicOr(&bits[r >> 5], 1u << (r & 31));
                    }
                    __syncwarp();
                    F = L;
                }
            }
        } else {
            // rows beyond the bitmap: one column at a time, lane q testing the
            // q-th entry of the exact prefix
            for (int j = 0; j < p; j++) {
                const Cand *pre = mrg + j;  // entry e at pre[e * p]
                const int ex = mlen[j];
                const int rq = lane < ex ? pre[(size_t)lane * p].row : -1;
                const bool taken = rq >= 0 && hash_has(hset, rq);
                const unsigned bal = __ballot_sync(0xffffffffu, rq >= 0 && !taken);
                int r = -1;
                if (bal != 0) {
                    r = __shfl_sync(0xffffffffu, rq, __ffs(bal) - 1);
                } else {
                    if (lane == 0) r = walk(j);
                    r = __shfl_sync(0xffffffffu, r, 0);
                }
                if (lane == 0) {
                    chosen[j] = r;
                    if (r >= 0) hash_put(hset, r);
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    if (C != nullptr)
        for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
            const int j = idx / p, k = idx % p;
            const int r = chosen[j];
            C[idx] = (r >= 0) ? A21[(int64_t)k * lda + r] : 0.0;
        }
    if (rows_out != nullptr)
        for (int j = threadIdx.x; j < p; j += blockDim.x) rows_out[j] = chosen[j];
}

// C(j, :) = A21(rows[j], :) (zero where rows[j] < 0), row-major
__global__ void k_gather_rows(const double *__restrict__ A21, int64_t lda, int p,
                              const int32_t *__restrict__ rows, double *__restrict__ C) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < p * p; idx += gridDim.x * blockDim.x) {
        const int j = idx / p, k = idx % p;
        const int r = rows[j];
        C[idx] = (r >= 0) ? A21[(int64_t)k * lda + r] : 0.0;
    }
}

}  // namespace

// Rows per block of pass 1: the largest B = 2^lg <= 64 with ceil(m / B) >=
// min(m, p), so that every column has at least K_j block maxima.
int relaxed_block_lg(int64_t m, int p) {
    const int64_t need = m < p ? m : p;
    int lg = 6;
    while (lg > 0 && ((m + (1LL << lg) - 1) >> lg) < need) lg--;
    return lg;
}

static size_t relaxed_head_bytes(int p) {
    // candidate lists (one per column), their lengths, the chosen rows
    const size_t b = sizeof(Cand) * (size_t)p * p + sizeof(int) * (size_t)p + sizeof(int32_t) * (size_t)p;
    return (b + 255) & ~(size_t)255;
}

size_t relaxed_aux_bytes(int64_t m, int p, int /*num_sms*/) {
    const int lg = relaxed_block_lg(m, p);
    const int64_t nb = m > 0 ? (m + (1LL << lg) - 1) >> lg : 0;
    return relaxed_head_bytes(p) + sizeof(unsigned long long) * (size_t)p * (size_t)nb;  // + block maxima
}

// TMA map of A21 (m x p column-major, lda) in boxes of 64 rows x 32 columns,
// unswizzled (each column's rows contiguous); false when A21 does not allow one
static bool make_map_bm(CUtensorMap *map, const double *A21, int64_t m, int p, int64_t lda) {
    if ((reinterpret_cast<uintptr_t>(A21) & 15) != 0 || ((lda * 8) & 15) != 0) return false;
    if (m >= ((int64_t)1 << 31)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tc::encode_fn();
    if (enc == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)p};
    cuuint64_t strides[1] = {(cuuint64_t)lda * 8};
    cuuint32_t box[2] = {(cuuint32_t)kBmR, (cuuint32_t)kBmC};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(A21), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static size_t greedy_smem(int p, int nslot, int rmax) {
    return sizeof(Cand) * (size_t)p * nslot * greedy_head(nslot) + sizeof(int) * (size_t)p +
           sizeof(unsigned) * (size_t)((rmax + 31) / 32);
}

cudaError_t launch_compress_relaxed(const double *A21, int64_t m, int p, int64_t lda, double *C,
                                    int32_t *rows, void *aux, int32_t *info, int num_sms,
                                    cudaStream_t st) {
    Cand *lists = reinterpret_cast<Cand *>(aux);
    int *lens = reinterpret_cast<int *>(lists + (size_t)p * p);
    int32_t *chosen = reinterpret_cast<int32_t *>(lens + p);
    unsigned long long *bmax = reinterpret_cast<unsigned long long *>(static_cast<char *>(aux) + relaxed_head_bytes(p));
    if (m > 0) {
        const int lg = relaxed_block_lg(m, p);
        const int64_t nb = (m + (1LL << lg) - 1) >> lg;
        // pass 1: a persistent grid, eight CTAs of 256 threads per SM at most
        const int64_t units = ((m + 63) >> 6) * p;
        int64_t g1 = (units + 31) / 32;
        if (g1 > 8LL * num_sms) g1 = 8LL * num_sms;
        const bool vec = (reinterpret_cast<uintptr_t>(A21) & 15) == 0 && (lda & 1) == 0;
        CUtensorMap map;
        if (lg == 6 && vec && make_map_bm(&map, A21, m, p, lda)) {
            const size_t smem = (size_t)kBmStages * kBmR * kBmC * 8 + 1024;
            cudaError_t e = smem_at_least((const void *)k_block_max_tma, smem);
            if (e != cudaSuccess) return e;
            const int64_t ntiles = ((m + kBmR - 1) / kBmR) * ((p + kBmC - 1) / kBmC);
            int64_t g = 2LL * num_sms;
            if (g > ntiles) g = ntiles;
            k_block_max_tma<<<(unsigned)g, kBmThreads, smem, st>>>(map, m, p, nb, bmax, info);
        } else if (vec && lg == 6)
            k_block_max<true, true><<<(unsigned)g1, 256, 0, st>>>(A21, m, p, lda, lg, nb, bmax, info);
        else if (lg == 6)
            k_block_max<false, true><<<(unsigned)g1, 256, 0, st>>>(A21, m, p, lda, lg, nb, bmax, info);
        else if (vec)
            k_block_max<true, false><<<(unsigned)g1, 256, 0, st>>>(A21, m, p, lda, lg, nb, bmax, info);
        else
            k_block_max<false, false><<<(unsigned)g1, 256, 0, st>>>(A21, m, p, lda, lg, nb, bmax, info);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        // pass 2: one CTA per column
        const size_t smem = (sizeof(unsigned long long) + sizeof(int)) * kCap;
        err = smem_at_least((const void *)k_relaxed_pick, smem);
        if (err != cudaSuccess) return err;
        k_relaxed_pick<<<p, kT1, smem, st>>>(A21, m, p, lda, lg, nb, bmax, 0, 1, 0, lists, lens, info);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    } else {
        cudaError_t err = cudaMemsetAsync(lens, 0, sizeof(int) * (size_t)p, st);
        if (err != cudaSuccess) return err;
    }
    // pass 3: the greedy (one CTA) picks the rows; pass 4: the gather of those
    // rows into C (p^2 scattered reads) runs over many CTAs so that the reads overlap
    const int rmax = m <= kBitmapRows ? (int)m : 0;
    const size_t gsmem = greedy_smem(p, 1, rmax);
    cudaError_t err2 = smem_at_least((const void *)k_relaxed_greedy, gsmem);
    if (err2 != cudaSuccess) return err2;
    k_relaxed_greedy<<<1, kGreedyThreads, gsmem, st>>>(nullptr, 0, p, 1, lists, lens, nullptr, chosen, rmax);
    err2 = cudaGetLastError();
    if (err2 != cudaSuccess) return err2;
    k_gather_rows<<<(p * p + 255) / 256, 256, 0, st>>>(A21, lda, p, chosen, C);
    err2 = cudaGetLastError();
    if (err2 != cudaSuccess || rows == nullptr) return err2;
    return cudaMemcpyAsync(rows, chosen, sizeof(int32_t) * (size_t)p, cudaMemcpyDeviceToDevice, st);
}

size_t relaxed_candidate_bytes(int nslot, int p) {
    return sizeof(Cand) * (size_t)p * nslot * p + sizeof(int) * (size_t)p * nslot;
}

// Row split (Section 6): the candidate lists of one row block of A21 (one
// segment), into slot `slot` of `nslot`.
cudaError_t launch_relaxed_candidates(const double *A21, int64_t m, int p, int64_t lda, int row0, int slot,
                                      int nslot, void *cand, int32_t *info, cudaStream_t st) {
    Cand *lists = reinterpret_cast<Cand *>(cand);
    int *lens = reinterpret_cast<int *>(lists + (size_t)p * nslot * p);
    if (m == 0) {
        // an empty block contributes empty lists
        for (int j = 0; j < p; j++) {
            cudaError_t e = cudaMemsetAsync(lens + (size_t)j * nslot + slot, 0, sizeof(int), st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const size_t smem = (sizeof(unsigned long long) + sizeof(int)) * kCap;
    cudaError_t err = smem_at_least((const void *)k_relaxed_topk, smem);
    if (err != cudaSuccess) return err;
    k_relaxed_topk<<<p, kT1, smem, st>>>(A21, m, p, lda, slot, nslot, row0, lists, lens, info);
    return cudaGetLastError();
}

// The greedy over the nslot lists of every column; rows[j] = the chosen A21
// row of C row j (-1: none).  C is not written.
cudaError_t launch_relaxed_select(int p, int nslot, const void *cand, int32_t *rows, cudaStream_t st) {
    const Cand *lists = reinterpret_cast<const Cand *>(cand);
    const int *lens = reinterpret_cast<const int *>(lists + (size_t)p * nslot * p);
    const size_t gsmem = greedy_smem(p, nslot, 0);
    cudaError_t err = smem_at_least((const void *)k_relaxed_greedy, gsmem);
    if (err != cudaSuccess) return err;
    k_relaxed_greedy<<<1, kGreedyThreads, gsmem, st>>>(nullptr, 0, p, nslot, lists, lens, nullptr, rows, 0);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double *A21, int64_t lda, int p, const int32_t *rows, double *C,
                               cudaStream_t st) {
    k_gather_rows<<<(p * p + 255) / 256, 256, 0, st>>>(A21, lda, p, rows, C);
    return cudaGetLastError();
}

}  // namespace ctp
