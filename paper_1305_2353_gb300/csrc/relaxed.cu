// relaxed.cu -- K2: relaxed compression of A21 (Section 4.2).
//
// The paper's construction is sequential: for j = 1..p, the unflagged row with
// the largest |a21(i,j)| (lowest row on ties) is flagged and copied into row j
// of C.  Before column j at most j-1 rows are flagged, so its choice is always
// among the j largest entries of column j in the order (|a| desc, row asc).  The
// GPU form is therefore exact and one-pass:
//   phase 1  (HBM-bound) each CTA streams one contiguous segment of one column
//            and keeps the top K_j = j+1 entries of that segment: values that
//            beat the current K-th best are appended to a shared buffer, which
//            is compacted by a bitonic sort whenever it fills (rarely: for
//            random data a handful of times per segment);
//   phase 2  one CTA runs the paper's greedy: for each column it merges the
//            sorted segment lists and takes the first unflagged row;
//   phase 3  the chosen rows are gathered, with their signs, into C.
// Magnitudes are compared as integer keys (sign bit cleared), so no FP64
// arithmetic is involved and the result is bit-exact.
#include "ctp_internal.cuh"

namespace ctp {

namespace {

constexpr int kT1 = 512;      // threads per CTA in phase 1
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
// memory: exact, and no sort.  Every thread passes its own keys through
// `each(f)` (f(key) is called once per key it holds).
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
        each([&](unsigned long long v) {
            if ((v & mask) == prefix) atomicAdd(&rs.hist[(v >> shift) & 255u], 1u);
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

// Phase 1: CTA (seg, j) keeps the top K_j entries of rows [seg*L, (seg+1)*L) of
// column j.  Its list goes to slot s = seg_base + seg of nslot lists per column;
// rows are reported as row0 + (row in A21) (row0 > 0 when A21 is one row block
// of a larger matrix).
// The stream is HBM-bound: each pass reads kChunk rows, four per thread in
// flight.  A threshold thr (a lower bound of the K-th largest key of the
// segment, taken as the K-th largest of what was seen so far by radix
// selection) filters the stream, so only entries >= thr reach the shared
// buffer (ties kept: a superset of the top K); when the buffer fills, the
// threshold is raised and the buffer filtered again.  At the end the survivors
// (K plus ties) are sorted once into the paper's order (|a| descending, lower
// row first).
__global__ void __launch_bounds__(kT1)
    k_relaxed_topk(const double *__restrict__ A21, int64_t m, int p, int64_t lda, int64_t L,
                   int seg_base, int nslot, int row0, Cand *__restrict__ lists, int *__restrict__ lens,
                   int32_t *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *key = reinterpret_cast<unsigned long long *>(smraw);  // [kCap]
    int *row = reinterpret_cast<int *>(key + kCap);                           // [kCap]
    __shared__ int cnt;
    __shared__ int wsum[kT1 / 32 + 1];
    __shared__ RadixScratch rs;
    const int j = blockIdx.y, seg = blockIdx.x;
    const int64_t r0 = (int64_t)seg * L, r1 = (r0 + L < m) ? r0 + L : m;
    const int64_t len = r1 > r0 ? r1 - r0 : 0;
    const int K = (int)((int64_t)j + 1 < len ? (int64_t)j + 1 : len);
    const double *col = A21 + (int64_t)j * lda;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    bool nonfinite = false;
    bool have_thr = false;
    // thr: the K-th largest key among the rows seen so far.  A later row whose
    // key equals it ranks after every earlier tie (rows only grow along the
    // stream), so it cannot enter the top K: later rows need key > thr.
    unsigned long long thr = 0;
    auto buffer_each = [&](auto f) {
        for (int i = threadIdx.x; i < cnt; i += kT1) f(key[i]);
    };
    constexpr int kPer = kChunk / kT1;
    // the next chunk's loads are issued before this chunk is processed, so one
    // chunk is always in flight per thread
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
                for (int q = 0; q < kPer; q++)
                    if (base + q * kT1 + threadIdx.x < r1) f(kv[q]);
            });
            have_thr = true;
            fresh = true;
        }
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const int64_t r = base + q * kT1 + threadIdx.x;
            const bool keep = r < r1 && (!have_thr || kv[q] > thr || (fresh && kv[q] == thr));
            warp_append(keep, kv[q], (int)r, key, row, &cnt);
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
    const int k = n < K ? n : K;
    const int slot = j * nslot + seg_base + seg;
    Cand *out = lists + (int64_t)slot * p;
    for (int i = threadIdx.x; i < k; i += kT1) {
        Cand c;
        c.key = key[i];
        c.row = row0 + row[i];
        c.pad = 0;
        out[i] = c;
    }
    if (threadIdx.x == 0) lens[slot] = k;
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
}

// Phases 2 and 3: the greedy of Section 4.2 over the merged candidate lists,
// then the gather of the chosen rows into C (row-major, signed).
//   (a) every thread merges, for one column, the first kHead entries of each
//       segment list into one sorted prefix; the prefix is exact up to the
//       smallest staged entry of any segment that holds more than kHead;
//   (b) one thread runs the sequential greedy over those prefixes, with the
//       chosen rows in a small open-addressing hash set; a column that
//       exhausts its exact prefix (many collisions) falls back to walking the
//       full segment lists in global memory.
constexpr int kHead = 4;
constexpr int kHash = 1024;  // > 2 * kMaxP slots

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

__global__ void __launch_bounds__(256)
    k_relaxed_greedy(const double *__restrict__ A21, int64_t lda, int p, int nseg,
                     const Cand *__restrict__ lists, const int *__restrict__ lens,
                     double *__restrict__ C, int32_t *__restrict__ rows_out) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int W = nseg * kHead;                                      // merged prefix width
    Cand *mrg = reinterpret_cast<Cand *>(gsm);                       // [p][W]
    int *mlen = reinterpret_cast<int *>(mrg + (size_t)p * W);        // [p] exact prefix length
    __shared__ int chosen[kMaxP];
    __shared__ int hset[kHash];
    for (int i = threadIdx.x; i < kHash; i += blockDim.x) hset[i] = -1;
    // (a) per-column merge of the staged heads
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        Cand *out = mrg + (size_t)j * W;
        int cnt = 0;
        bool have_lim = false;
        Cand lim;
        lim.key = 0;
        lim.row = 0x7fffffff;
        for (int s = 0; s < nseg; s++) {
            const int li = j * nseg + s;
            const int len = lens[li];
            const int h = len < kHead ? len : kHead;
            for (int q = 0; q < h; q++) {
                const Cand c = lists[(int64_t)li * p + q];
                int at = cnt++;
                while (at > 0 && before(c, out[at - 1])) {  // insertion into the sorted prefix
                    out[at] = out[at - 1];
                    --at;
                }
                out[at] = c;
            }
            if (len > kHead) {
                // entries beyond this segment's staged ones may come after its last staged entry
                const Cand last = lists[(int64_t)li * p + kHead - 1];
                if (!have_lim || before(last, lim)) {
                    lim = last;
                    have_lim = true;
                }
            }
        }
        int exact = cnt;
        if (have_lim) {
            exact = 0;
            while (exact < cnt && !before(lim, out[exact])) ++exact;  // out[exact] <= lim in order
        }
        mlen[j] = exact;
    }
    __syncthreads();
    // (b) the sequential greedy
    if (threadIdx.x == 0) {
        for (int j = 0; j < p; j++) {
            const Cand *pre = mrg + (size_t)j * W;
            const int ex = mlen[j];
            int r = -1;
            bool done = false;
            for (int q = 0; q < ex; q++)
                if (!hash_has(hset, pre[q].row)) {
                    r = pre[q].row;
                    done = true;
                    break;
                }
            if (!done) {
                // slow path: walk the full segment lists of column j in order
                int head[64];
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
                    if (bs < 0) break;  // every A21 row is already flagged
                    if (!hash_has(hset, best.row)) {
                        r = best.row;
                        break;
                    }
                    head[bs]++;
                }
            }
            chosen[j] = r;
            if (r >= 0) hash_put(hset, r);
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

size_t relaxed_aux_bytes(int64_t m, int p, int num_sms) {
    const int nseg = relaxed_segments(m, p, num_sms);
    // candidate lists, their lengths, the chosen rows
    return sizeof(Cand) * (size_t)p * nseg * p + sizeof(int) * (size_t)p * nseg + sizeof(int32_t) * (size_t)p;
}

int relaxed_segments(int64_t m, int p, int num_sms) {
    // enough CTAs to cover the SMs several times, segments of at least 8 chunks
    int64_t want = (8LL * num_sms + p - 1) / p;
    int64_t maxseg = (m + 8 * kChunk - 1) / (8 * kChunk);
    int64_t s = want < maxseg ? want : maxseg;
    if (s < 1) s = 1;
    if (s > 8) s = 8;  // the greedy stages 4 heads of every list in shared memory
    return (int)s;
}

cudaError_t launch_compress_relaxed(const double *A21, int64_t m, int p, int64_t lda, double *C,
                                    int32_t *rows, void *aux, int32_t *info, int num_sms,
                                    cudaStream_t st) {
    const int nseg = relaxed_segments(m, p, num_sms);
    Cand *lists = reinterpret_cast<Cand *>(aux);
    int *lens = reinterpret_cast<int *>(lists + (size_t)p * nseg * p);
    if (m > 0) {
        const int64_t L = (m + nseg - 1) / nseg;
        const size_t smem = (sizeof(unsigned long long) + sizeof(int)) * kCap;
        cudaError_t err =
            smem_at_least((const void *)k_relaxed_topk, smem);
        if (err != cudaSuccess) return err;
        dim3 grid(nseg, p);
        k_relaxed_topk<<<grid, kT1, smem, st>>>(A21, m, p, lda, L, 0, nseg, 0, lists, lens, info);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    } else {
        cudaError_t err = cudaMemsetAsync(lens, 0, sizeof(int) * (size_t)p * nseg, st);
        if (err != cudaSuccess) return err;
    }
    // the greedy (one CTA) picks the rows; the gather of those rows into C (p^2
    // scattered reads) runs over many CTAs so that the reads overlap
    const size_t gsmem = sizeof(Cand) * (size_t)p * nseg * kHead + sizeof(int) * (size_t)p;
    cudaError_t err2 =
        smem_at_least((const void *)k_relaxed_greedy, gsmem);
    if (err2 != cudaSuccess) return err2;
    int32_t *chosen = reinterpret_cast<int32_t *>(lens + (size_t)p * nseg);
    k_relaxed_greedy<<<1, 256, gsmem, st>>>(nullptr, 0, p, nseg, lists, lens, nullptr, chosen);
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
    k_relaxed_topk<<<dim3(1, p), kT1, smem, st>>>(A21, m, p, lda, m, slot, nslot, row0, lists, lens, info);
    return cudaGetLastError();
}

// The greedy over the nslot lists of every column; rows[j] = the chosen A21
// row of C row j (-1: none).  C is not written.
cudaError_t launch_relaxed_select(int p, int nslot, const void *cand, int32_t *rows, cudaStream_t st) {
    const Cand *lists = reinterpret_cast<const Cand *>(cand);
    const int *lens = reinterpret_cast<const int *>(lists + (size_t)p * nslot * p);
    const size_t gsmem = sizeof(Cand) * (size_t)p * nslot * kHead + sizeof(int) * (size_t)p;
    cudaError_t err = smem_at_least((const void *)k_relaxed_greedy, gsmem);
    if (err != cudaSuccess) return err;
    k_relaxed_greedy<<<1, 256, gsmem, st>>>(nullptr, 0, p, nslot, lists, lens, nullptr, rows);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double *A21, int64_t lda, int p, const int32_t *rows, double *C,
                               cudaStream_t st) {
    k_gather_rows<<<(p * p + 255) / 256, 256, 0, st>>>(A21, lda, p, rows, C);
    return cudaGetLastError();
}

}  // namespace ctp
