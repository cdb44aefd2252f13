// Spatial ordering and packing of the sources for the near-field kernels.
//
// FP32C needs sources grouped into compact chunks so that float32 offsets from a
// per-chunk float64 origin keep the precision of close pairs.  The charges are
// ordered along the Hilbert curve of a 256^3 grid over the box (hilbert_key24) by a
// stable least-significant-digit radix sort (8-bit digits), then packed 128 at
// a time with the midpoint of each chunk's bounding box as its origin.
#include "psum_internal.cuh"

namespace psum {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerThread = 8;
constexpr int kSortTile = kSortThreads * kSortPerThread;   // 2048 keys per block
constexpr int kRadix = 256;

__global__ void k_curve_keys(const double* __restrict__ x, int64_t n, double d0, double d1, double d2,
                         uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dd[3] = {d0, d1, d2};
    uint32_t c[3];
    for (int k = 0; k < 3; ++k) {
        double u = (x[3 * i + k] / dd[k] + 0.5) * 256.0;
        int v = (int)floor(u);
        v = v < 0 ? 0 : (v > 255 ? 255 : v);      // also maps NaN (validated elsewhere) into range
        c[k] = (uint32_t)v;
    }
    keys[i] = hilbert_key24(c[0], c[1], c[2]);
    vals[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                            uint32_t* __restrict__ hist, int nblk) {
    __shared__ uint32_t cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortPerThread; ++k) {
        const int64_t i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[(int64_t)d * nblk + blockIdx.x] = cnt[d];
}

// exclusive scan of `total` counts in place, one block of 1024 threads
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* __restrict__ hist, int64_t total) {
    __shared__ uint32_t s[1024];
    const int64_t per = (total + 1023) / 1024;
    const int64_t b = threadIdx.x * per;
    const int64_t e = b + per < total ? b + per : total;
    uint32_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += hist[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const uint32_t v = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - sum;
    for (int64_t i = b; i < e; ++i) {
        const uint32_t v = hist[i];
        hist[i] = run;
        run += v;
    }
}

// Stable scatter: warp w of block b owns keys [b*T + w*256, +256) and walks them in
// order, 32 at a time; equal digits inside a step are ranked by lane.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin, int64_t n, int shift,
                                                               const uint32_t* __restrict__ offs, int nblk,
                                                               uint32_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout) {
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kSortTile + w * (kSortPerThread * 32);
    for (int k = 0; k < kSortPerThread; ++k) {
        const int64_t i = wbase + k * 32 + lane;
        if (i < n) atomicAdd(&wcnt[w][(kin[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t run = offs[(int64_t)d * nblk + blockIdx.x];
        for (int ww = 0; ww < kSortWarps; ++ww) {
            const uint32_t c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (int k = 0; k < kSortPerThread; ++k) {
        const int64_t i = wbase + k * 32 + lane;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t dig = valid ? ((key >> shift) & (kRadix - 1)) : (uint32_t)(kRadix + lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, dig);
        const uint32_t rank = __popc(peers & lt);
        uint32_t pos = 0;
        if (valid) pos = wcnt[w][dig] + rank;
        __syncwarp();
        if (valid && rank == 0) wcnt[w][dig] += __popc(peers);
        __syncwarp();
        if (valid) {
            kout[pos] = key;
            vout[pos] = vin[i];
        }
    }
}

// One warp per group of kNearChunk sorted positions: the bounding-box midpoint is the
// float64 origin, stored with the group radius (largest distance of a point from it);
// each point's offset from the origin is split into a float32 hi part and the float32
// rounding remainder lo, packed two float4 each: (x,x,y,y),(z,z,q,q) and (xl,xl,yl,yl),(zl,zl,ql,ql)
// (ql = q - float(q), read only by the float-float kernels).
// Padding points (s >= n) get q = 0 and a far-away position.  `ext` (optional) receives each
// group's bounding-box half extents about its origin.
// With a group table (batches) group g covers the sorted positions
// [grp_start[g], grp_start[g] + grp_count[g]); without one, [128 g, min(128 (g+1), n)).
constexpr int kPackWarps = 16;  // warps (groups) per block of k_pack32

__global__ void __launch_bounds__(32 * kPackWarps) k_pack32(const double* __restrict__ x, const double* __restrict__ q,
                         const uint32_t* __restrict__ perm, int64_t n, int64_t n_groups,
                         const int64_t* __restrict__ grp_start, const int* __restrict__ grp_count,
                         float4* __restrict__ pk_hi, float4* __restrict__ pk_lo, double* __restrict__ org,
                         double* __restrict__ xs, float4* __restrict__ ext) {
    const int64_t grp = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const bool live = grp < n_groups;      // a warp past the last group takes part in the barriers only
    const int64_t s0 = !live ? 0 : grp_start ? grp_start[grp] : grp * kNearChunk;
    const int64_t s1 = !live ? 0 : grp_start ? s0 + grp_count[grp] : (grp + 1) * kNearChunk < n ? (grp + 1) * kNearChunk : n;
    constexpr int per = kNearChunk / 32;
    double px[per][3], pq[per];
    bool ok[per];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int64_t s = s0 + k * 32 + lane;
        ok[k] = s < s1;
        if (ok[k]) {
            const int64_t i = perm ? (int64_t)perm[s] : s;
            for (int c = 0; c < 3; ++c) {
                px[k][c] = x[3 * i + c];
                lo[c] = fmin(lo[c], px[k][c]);
                hi[c] = fmax(hi[c], px[k][c]);
            }
            pq[k] = q ? q[i] : 0.0;               // no charges: a pack of evaluation points
        }
    }
    double o[3];
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], off));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], off));
        }
        o[c] = lo[c] <= hi[c] ? 0.5 * (lo[c] + hi[c]) : 0.0;
    }
    // float32 charges with the rounding error diffused along the group (in sorted order):
    // each charge absorbs the error carried so far, so the group's float32 charges sum to
    // its float64 total up to one rounding; a non-neutral rounding residue would add the
    // potential of a net charge over all images to every target.
    // The recurrence is sequential, a chain of float64 operations over the group's charges
    // staged in shared memory.  The block's groups run theirs side by side, one lane each of
    // its first warp: a float64 warp instruction occupies the SM's narrow float64 pipe the same
    // time however few lanes it has, so one lane per warp would cost kPackWarps times as much.
    // (Rows padded by one element: the lanes' rows fall in different banks.)
    __shared__ double s_q[kPackWarps][kNearChunk + 1];
    __shared__ float s_f[kPackWarps][kNearChunk + 1];
    __shared__ int s_cnt[kPackWarps];
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < per; ++k) s_q[w][k * 32 + lane] = ok[k] ? pq[k] : 0.0;
    if (lane == 0) s_cnt[w] = (int)(s1 - s0);
    __syncthreads();
    if (threadIdx.x < kPackWarps) {
        const int wg = threadIdx.x;
        const int cnt = s_cnt[wg];
        double carry = 0.0;
        for (int m = 0; m < cnt; ++m) {
            const double qm = s_q[wg][m];
            const float v = (float)(qm - carry);
            carry += (double)v - qm;
            s_f[wg][m] = v;
        }
    }
    __syncthreads();
    if (!live) return;
    float fqk[per];
#pragma unroll
    for (int k = 0; k < per; ++k) fqk[k] = s_f[w][k * 32 + lane];
    double r2max = 0.0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int64_t s = grp * kNearChunk + k * 32 + lane;
        float fx = 1.0e3f, fy = 1.0e3f, fz = 1.0e3f, fq = 0.f, lx = 0.f, ly = 0.f, lz = 0.f, lq = 0.f;
        if (ok[k]) {
            const double rx = px[k][0] - o[0], ry = px[k][1] - o[1], rz = px[k][2] - o[2];
            r2max = fmax(r2max, rx * rx + ry * ry + rz * rz);
            fx = (float)rx; fy = (float)ry; fz = (float)rz;
            lx = (float)(rx - (double)fx); ly = (float)(ry - (double)fy); lz = (float)(rz - (double)fz);
            fq = fqk[k];
            lq = (float)(pq[k] - (double)fq);     // the charge's float-float remainder (FF pair sums)
        }
        pk_hi[2 * s] = make_float4(fx, fx, fy, fy);
        pk_hi[2 * s + 1] = make_float4(fz, fz, fq, fq);
        pk_lo[2 * s] = make_float4(lx, lx, ly, ly);
        pk_lo[2 * s + 1] = make_float4(lz, lz, lq, lq);
        if (xs) {
            xs[3 * s] = ok[k] ? px[k][0] : 1.0e3;
            xs[3 * s + 1] = ok[k] ? px[k][1] : 1.0e3;
            xs[3 * s + 2] = ok[k] ? px[k][2] : 1.0e3;
        }
    }
    for (int off = 16; off > 0; off >>= 1) r2max = fmax(r2max, __shfl_xor_sync(0xffffffffu, r2max, off));
    if (lane == 0) {
        org[4 * grp] = o[0]; org[4 * grp + 1] = o[1]; org[4 * grp + 2] = o[2];
        org[4 * grp + 3] = sqrt(r2max);
        if (ext) {
            // half extents of the bounding box about the origin, rounded up (never smaller)
            float h[3];
            for (int c = 0; c < 3; ++c) h[c] = lo[c] <= hi[c] ? __double2float_ru(fmax(hi[c] - o[c], o[c] - lo[c])) : 0.f;
            ext[grp] = make_float4(h[0], h[1], h[2], 0.f);
        }
    }
}

__global__ void k_pack64(const double* __restrict__ x, const double* __restrict__ q, int64_t n, int64_t n_pad,
                         double4_32a* __restrict__ pk) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    if (s < n)
        pk[s] = make_double4_32a(x[3 * s], x[3 * s + 1], x[3 * s + 2], q ? q[s] : 0.0);
    else
        pk[s] = make_double4_32a(1.0e3, 1.0e3, 1.0e3, 0.0);
}

// batches: packed point s of group g = s / 128 holds charge grp_start[g] + s % 128 if
// s % 128 < grp_count[g] (caller order inside each system), padding otherwise
__global__ void k_pack64_groups(const double* __restrict__ x, const double* __restrict__ q, int64_t n_pts,
                                const int64_t* __restrict__ grp_start, const int* __restrict__ grp_count,
                                double4_32a* __restrict__ pk) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pts) return;
    const int64_t g = s / kNearChunk;
    const int k = (int)(s - g * kNearChunk);
    if (k < grp_count[g]) {
        const int64_t i = grp_start[g] + k;
        pk[s] = make_double4_32a(x[3 * i], x[3 * i + 1], x[3 * i + 2], q[i]);
    } else {
        pk[s] = make_double4_32a(1.0e3, 1.0e3, 1.0e3, 0.0);
    }
}

cudaError_t launch_pack64_groups(const double* x, const double* q, int64_t n_pts, const int64_t* grp_start,
                                 const int* grp_count, double4_32a* pk, cudaStream_t st) {
    k_pack64_groups<<<(unsigned)((n_pts + 255) / 256), 256, 0, st>>>(x, q, n_pts, grp_start, grp_count, pk);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
int sort_blocks(int64_t n) { return (int)((n + kSortTile - 1) / kSortTile); }

// Stable LSD radix sort of (key, value) pairs, 8 bits per pass over `passes` passes,
// ping-ponging (ka, va) -> (kb, vb) -> ...: the result ends in (ka, va) after an even
// number of passes and in (kb, vb) after an odd one; hist is scratch.
cudaError_t launch_radix_sort(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, uint32_t* hist, int64_t n,
                              int passes, cudaStream_t st) {
    const int nblk = sort_blocks(n);
    uint32_t *ki = ka, *vi = va, *ko = kb, *vo = vb;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        k_sort_hist<<<nblk, kSortThreads, 0, st>>>(ki, n, shift, hist, nblk);
        k_sort_scan<<<1, 1024, 0, st>>>(hist, (int64_t)kRadix * nblk);
        k_sort_scatter<<<nblk, kSortThreads, 0, st>>>(ki, vi, n, shift, hist, nblk, ko, vo);
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    return cudaGetLastError();
}

// Small inputs in one block: the (key, index) pairs as 64-bit words in shared memory, a
// bitonic sort, the same order as the stable radix sort (ties broken by the index), in one
// launch instead of nine.
constexpr int kSmallSort = 4096;
constexpr int kSmallSortThreads = 1024;

__global__ void __launch_bounds__(kSmallSortThreads) k_sort_small(const uint32_t* __restrict__ kin,
                                                                  const uint32_t* __restrict__ vin, int n,
                                                                  uint32_t* __restrict__ kout,
                                                                  uint32_t* __restrict__ vout) {
    __shared__ unsigned long long w[kSmallSort];
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += kSmallSortThreads)
        w[i] = i < n ? ((unsigned long long)kin[i] << 32) | vin[i] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += kSmallSortThreads) {
                const int p = i ^ j;
                if (p > i) {
                    const unsigned long long a = w[i], b = w[p];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        w[i] = b;
                        w[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += kSmallSortThreads) {
        kout[i] = (uint32_t)(w[i] >> 32);
        vout[i] = (uint32_t)(w[i] & 0xffffffffu);
    }
}

int curve_sort_launches(int64_t n) { return n <= kSmallSort ? 2 : 1 + 3 * 3; }

// Hilbert order of the points: 24-bit keys, written to (kb, vb) and sorted (3 radix passes,
// or one block for small inputs) so that the sorted keys and the permutation end in (ka, va).
cudaError_t launch_curve_sort(const double* x, int64_t n, const double d[3], uint32_t* ka, uint32_t* va,
                               uint32_t* kb, uint32_t* vb, uint32_t* hist, cudaStream_t st) {
    const int bs = 256;
    k_curve_keys<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(x, n, d[0], d[1], d[2], kb, vb);
    if (n <= kSmallSort) {
        k_sort_small<<<1, kSmallSortThreads, 0, st>>>(kb, vb, (int)n, ka, va);
        return cudaGetLastError();
    }
    return launch_radix_sort(kb, vb, ka, va, hist, n, 3, st);
}

cudaError_t launch_pack32(const double* x, const double* q, const uint32_t* perm, int64_t n, int64_t n_groups,
                          float4* pk_hi, float4* pk_lo, double* org, cudaStream_t st, double* xs, float4* ext) {
    const int warps = kPackWarps;
    k_pack32<<<(unsigned)((n_groups + warps - 1) / warps), 32 * warps, 0, st>>>(x, q, perm, n, n_groups, nullptr,
                                                                                  nullptr, pk_hi, pk_lo, org, xs, ext);
    return cudaGetLastError();
}

cudaError_t launch_pack32_groups(const double* x, const double* q, const uint32_t* perm, int64_t n_groups,
                                 const int64_t* grp_start, const int* grp_count, float4* pk_hi, float4* pk_lo,
                                 double* org, cudaStream_t st, float4* ext) {
    const int warps = kPackWarps;
    k_pack32<<<(unsigned)((n_groups + warps - 1) / warps), 32 * warps, 0, st>>>(x, q, perm, 0, n_groups, grp_start,
                                                                                  grp_count, pk_hi, pk_lo, org,
                                                                                  nullptr, ext);
    return cudaGetLastError();
}

cudaError_t launch_pack64(const double* x, const double* q, int64_t n, int64_t n_pad, double4_32a* pk, cudaStream_t st) {
    const int bs = 256;
    k_pack64<<<(unsigned)((n_pad + bs - 1) / bs), bs, 0, st>>>(x, q, n, n_pad, pk);
    return cudaGetLastError();
}

}  // namespace psum
