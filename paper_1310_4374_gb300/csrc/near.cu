// Near-field direct image sum (Sec. 2.1, Eq. 3; algorithm "get", steps 1 and 3):
//
//   phi_near(y)      = sum_{p in images} sum_i q_i / |y - x_i - p|       (K(0) = 0, Eq. 1)
//   grad phi_near(y) = sum_{p} sum_i q_i (x_i + p - y) / |y - x_i - p|^3
//
// at the N charges (potential and gradient), at the 2M check points (potential
// only), at the M check points as the partner difference of two image layers (potential
// only; each target's class selects its layer images and their weights +1, -1 or 0), or at
// separate evaluation points.  The kernels share one work decomposition:
//
//   * the work unit is (target tile, source chunk, image); the unit space is cut
//     into W equal contiguous work items (fixed, so every tile's partial-sum slots
//     and every summation order are fixed), which the resident CTAs take in order
//     from a device counter;
//   * a CTA stages a source chunk in shared memory once (bulk copies on an
//     mbarrier) and applies every image to it; the image shift is folded into the
//     targets in registers;
//   * a CTA writes each item's per-tile partial sums to the item's slot of a
//     partial buffer, and a reduction kernel adds the slots in a fixed order.
//
// FP32C: coordinates are float32 offsets from a float64 origin per group of
// 128 consecutive (Hilbert-sorted) points; the offset between a target group and
// a source chunk, minus the image vector, is formed in float64 and rounded once,
// so close pairs keep their relative precision.  Pair arithmetic uses packed
// f32x2 instructions on two targets at a time and MUFU rsqrt; per-unit float32
// partial sums are folded into a float32 (hi, lo) pair by Knuth's two-sum.
//
// FF: the same data in float-float arithmetic (hi + lo pairs) for float64-class
// results on the float32 pipe.
//
// FP64: absolute float64 coordinates; 1/sqrt(r^2) is a float32 MUFU estimate
// refined by one third-order step in float64.
//
// The charge sums (targets = sources) also have symmetric kernels, k_near32s (FP32C, FF)
// and k_near64s (FP64), which take each pair of tiles once with every image and add both
// the target's and the source's terms of a pair (near_sym.cu).
#include "near_common.cuh"

namespace psum {

struct Near32Args {
    const float4* src_hi;    // 2 float4 per source: (x,x,y,y),(z,z,q,q), offsets from the chunk origin
    const float4* src_lo;    // 2 float4 per source: (xl,xl,yl,yl),(zl,zl,0,0), the float32 rounding remainders
    const double* src_org;   // 4 per chunk: origin x, y, z and radius
    const float4* tgt_hi;    // same layouts for the targets (q unused)
    const float4* tgt_lo;
    const double* tgt_org;   // 4 per target group (kGroupsPerTile32 groups per tile)
    const double* shifts;    // image vectors, 3 per image, systems one after another
    double* partial;         // [tiles][max_contrib][4 or 1][kTile32]
    const double* src_x;     // float64 positions of the packed sources, 3 per point (ball trimming)
    double Rb;               // > 0: keep a source image x + p only if |x + p| <= Rb (get step 2)
    int64_t U, W;            // units, work items
    int* counter;            // next work item
    int* status;             // error words (kStatTimeout when a chunk copy never lands)
    int n_status;
    int inject;              // test hook: expect 16 bytes more than the copies bring
    int64_t limit;           // doubles of the partial buffer (debug bounds checks)
    int max_contrib, max_img;
    NearSysTable tab;
    // two-layer check sums (potential only): each target's class c (0..n_cls-1) rides in its
    // pack's charge slot; the image vector of (class c, image j) is shifts[shift0 + c n_img + j]
    // and its weight img_w[shift0 + c n_img + j]; grp_cls holds each target group's classes as
    // a bit mask.  n_cls = 1 and null tables: one image list, weight 1.
    const int* grp_cls;
    const double* grp_sub;       // [group][n_cls][4]: centre and radius of each class's points
    const float* img_w;
    int n_cls;
    // per source chunk (may be null): the first entry of its image list in `shifts` and its count
    // (units past the count add nothing); the backward's two-layer check sources
    const int* chunk_img0;
    const int* chunk_nimg;
};

// Two register budgets of the same kernel: 4 resident CTAs per SM (up to 128 registers) or
// 6 (80).  With work items handed out dynamically the larger budget, which lets the
// compiler keep more loads and rsqrt results in flight, is the faster one (109.8 against
// 115.7-121.1 ms for 1e5 charges); the batch autotuner times both.
constexpr int kNear32MinBlocks[2] = {4, 6};

template <bool kGrad, int kMinB, bool kTrim, bool kFF>
__global__ void __launch_bounds__(kThreads32, kMinB) k_near32(Near32Args a) {
    constexpr int NQ = kGrad ? 4 : 1;
    __shared__ float4 s_hi[2 * kNearChunk];
    __shared__ float4 s_lo[2 * kNearChunk];
    __shared__ float2 s_th[3][2][kThreads32];             // target hi offsets, [coord][pair]
    __shared__ float2 s_tl[kFF ? 3 : 1][2][kThreads32];   // FF: target lo offsets
    __shared__ float2 s_acc[NQ][2][2][kThreads32];        // [quantity][pair][hi, lo]
    // classes of the targets' image lists: 1, or (two-layer check sums) one per target
    const int ncls = kGrad ? 1 : a.n_cls;
    __shared__ int s_tcls[kGrad ? 1 : kTgt32][kThreads32];   // potential only: the targets' classes
    extern __shared__ float4 s_dyn4[];                    // [max_img][kTgt32][ncls][6] deltas, [max_img] flags,
    float* s_delta = (float*)s_dyn4;                      // potential only: [max_img][kTgt32][ncls] weights,
    int* s_near = (int*)(s_delta + 6 * kTgt32 * ncls * a.max_img);   // then (trimmed plans) the
    float* s_w = (float*)(s_near + a.max_img);            // compacted sources of a straddling unit
    constexpr int kWts = kGrad ? 0 : kTgt32;
    float4* s_hm = s_dyn4 + (6 * kTgt32 * ncls * a.max_img + a.max_img + kWts * ncls * a.max_img + 3) / 4;

    __shared__ int s_item;
    __shared__ int s_fail;
    __shared__ int s_wcnt[kThreads32 / 32];
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x;
    int64_t item = 0;
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        s_fail = 0;
    }
    __syncthreads();

    auto flush = [&](int64_t tile, int64_t first_unit) {
        const int64_t slot = item - sk_owner(first_unit, a.U, a.W);
        const int64_t off = ((tile * a.max_contrib + slot) * NQ) * kTile32;
        double* dst = a.partial + off;
        const bool ok = debug_in_range(off, NQ * kTile32, a.limit, a.status, a.n_status);
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi)
#pragma unroll
            for (int j = 0; j < 2 && ok; ++j) {
                const float2 h = s_acc[qi][j][0][tid], l = s_acc[qi][j][1][tid];
                dst[qi * kTile32 + (2 * j) * kThreads32 + tid] = (double)h.x + (double)l.x;
                dst[qi * kTile32 + (2 * j + 1) * kThreads32 + tid] = (double)h.y + (double)l.y;
            }
    };

    for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    item = s_item;
    __syncthreads();                     // every thread has the item before s_item changes
    if (item >= a.W) break;
    int64_t u = sk_bound(item, a.U, a.W);
    const int64_t u_end = sk_bound(item + 1, a.U, a.W);
    int sb = near_sys_by_unit(a.tab, u);
    int64_t cur_tile = -1, cur_chunk = -1, cur_first = 0;
    // two-layer check sums: a tile whose groups 2 and 3 hold no point (both marked
    // kGroupEmpty, the padding after the last points) runs its second packed target pair not at all
    bool pair1_live = true;
    while (u < u_end) {
        // the system descriptor is re-read (parameter or L1) rather than held in registers
        const NearSys* Sp = a.tab.many ? a.tab.many + sb : &a.tab.one;
        if (u >= Sp->unit0 + near_sys_units(*Sp)) {
            ++sb;
            continue;
        }
        const int n_img = Sp->n_img;
        const int64_t upt = Sp->n_chunks * n_img;
        const int64_t local = u - Sp->unit0;
        const int64_t tile_l = local / upt;
        const int64_t rem = local - tile_l * upt;
        const int64_t chunk_l = rem / n_img;
        const int img = (int)(rem - chunk_l * n_img);
        const int64_t tile = Sp->tile0 + tile_l;
        const int64_t chunk = Sp->src_chunk0 + (chunk_l * Sp->chunk_stride) % Sp->n_chunks;
        if (tile != cur_tile) {
            if (cur_tile >= 0) flush(cur_tile, cur_first);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int64_t i0 = (tile * kTgt32 + 2 * j) * kGroup + tid;
                const int64_t i1 = i0 + kGroup;
                const float4 A0 = a.tgt_hi[2 * i0], B0 = a.tgt_hi[2 * i0 + 1];
                const float4 A1 = a.tgt_hi[2 * i1], B1 = a.tgt_hi[2 * i1 + 1];
                s_th[0][j][tid] = make_float2(A0.x, A1.x);
                s_th[1][j][tid] = make_float2(A0.z, A1.z);
                s_th[2][j][tid] = make_float2(B0.x, B1.x);
                if constexpr (!kGrad) {
                    // a class outside 0..ncls-1 (the padding of a point-form pack holds 1e3
                    // there) reads class 0: the index stays inside the tables
                    const float c0 = B0.z, c1 = B1.z;
                    s_tcls[2 * j][tid] = ncls > 1 && c0 >= 0.f && c0 < (float)ncls ? (int)c0 : 0;
                    s_tcls[2 * j + 1][tid] = ncls > 1 && c1 >= 0.f && c1 < (float)ncls ? (int)c1 : 0;
                }
                if (kFF) {
                    const float4 C0 = a.tgt_lo[2 * i0], D0 = a.tgt_lo[2 * i0 + 1];
                    const float4 C1 = a.tgt_lo[2 * i1], D1 = a.tgt_lo[2 * i1 + 1];
                    s_tl[0][j][tid] = make_float2(C0.x, C1.x);
                    s_tl[kFF ? 1 : 0][j][tid] = make_float2(C0.z, C1.z);
                    s_tl[kFF ? 2 : 0][j][tid] = make_float2(D0.x, D1.x);
                }
#pragma unroll
                for (int qi = 0; qi < NQ; ++qi) {
                    s_acc[qi][j][0][tid] = make_float2(0.f, 0.f);
                    s_acc[qi][j][1][tid] = make_float2(0.f, 0.f);
                }
            }
            cur_tile = tile;
            cur_first = Sp->unit0 + tile_l * upt;
            pair1_live = kGrad || ncls <= 1 || !a.grp_cls ||
                         !(a.grp_cls[tile * kTgt32 + 2] & a.grp_cls[tile * kTgt32 + 3] & kGroupEmpty);
            cur_chunk = -1;
        }
        if (chunk != cur_chunk) {
            __syncthreads();   // every thread is done with the previous chunk, deltas and flags
            if (tid == 0) {
                // order this CTA's earlier shared-memory accesses before the copy engine's writes
                fence_proxy_async_smem();
                mbar_expect_tx(&s_bar, 2 * kChunkBytes + (a.inject ? 16 : 0));
                bulk_g2s(s_hi, a.src_hi + chunk * (2 * kNearChunk), kChunkBytes, &s_bar);
                bulk_g2s(s_lo, a.src_lo + chunk * (2 * kNearChunk), kChunkBytes, &s_bar);
            }
            const double* so = a.src_org + 4 * chunk;
            const int shift0 = Sp->shift0;
            // the item's units of this chunk are its images img .. im_hi - 1 (images innermost):
            // only those get offsets and classes
            const int im_lo = img;
            const int im_hi = (int)(u_end - u < (int64_t)(n_img - img) ? img + (u_end - u) : n_img);
            if (!kGrad && ncls > 1) {
                // per (image, group, class): the offset with the class's layer image, its
                // weight; a unit is near when a class present in a group is near
                for (int im = im_lo + tid; im < im_hi; im += kThreads32) s_near[im] = 0;
                __syncthreads();
                for (int e = im_lo * kTgt32 * ncls + tid; e < im_hi * kTgt32 * ncls; e += kThreads32) {
                    const int im = e / (kTgt32 * ncls), r = e - im * kTgt32 * ncls;
                    const int k = r / ncls, c = r - k * ncls;
                    // a class no target of the group has (padding included) is never read
                    if (!((a.grp_cls[cur_tile * kTgt32 + k] >> c) & 1)) continue;
                    const int ei = shift0 + c * n_img + im;
                    const double* sh = a.shifts + 3 * ei;
                    const double* to = a.tgt_org + 4 * (cur_tile * kTgt32 + k);
                    const double D0 = (to[0] - so[0]) - sh[0], D1 = (to[1] - so[1]) - sh[1],
                                 D2 = (to[2] - so[2]) - sh[2];
                    float* dl = s_delta + 6 * e;
                    dl[0] = (float)D0; dl[1] = (float)D1; dl[2] = (float)D2;
                    dl[3] = (float)(D0 - (double)dl[0]); dl[4] = (float)(D1 - (double)dl[1]);
                    dl[5] = (float)(D2 - (double)dl[2]);
                    s_w[e] = a.img_w[ei];
                    if (s_w[e] != 0.f) atomicOr(s_near + im, kUnitWeighted);
                    // the near test on the class's own points of the group
                    const double* sb = a.grp_sub + 4 * ((cur_tile * kTgt32 + k) * ncls + c);
                    const double E0 = (sb[0] - so[0]) - sh[0], E1 = (sb[1] - so[1]) - sh[1],
                                 E2 = (sb[2] - so[2]) - sh[2];
                    const double reach = kNearFactor * (sb[3] + so[3]);
                    if (E0 * E0 + E1 * E1 + E2 * E2 <= reach * reach)
                        atomicOr(s_near + im, k < 2 ? kUnitNear0 : kUnitNear1);
                }
                __syncthreads();
                // an image whose weight is zero for every class present (a padding layer image
                // of an anisotropic block) adds nothing to any target: skip its unit
                for (int im = im_lo + tid; im < im_hi; im += kThreads32)
                    s_near[im] = (s_near[im] & kUnitWeighted) ? (s_near[im] & ~kUnitWeighted) : kUnitOutside;
            } else
            for (int im = im_lo + tid; im < im_hi; im += kThreads32) {
                const int img0 = a.chunk_img0 ? a.chunk_img0[chunk] : shift0;
                const double* sh = a.shifts + 3 * (img0 + im);
                int nr = 0;
                bool weighted = false;
                for (int k = 0; k < kTgt32; ++k) {
                    const double* to = a.tgt_org + 4 * (cur_tile * kTgt32 + k);
                    const double* shk = sh;
                    if constexpr (!kGrad) {
                        const float wk = a.img_w ? a.img_w[shift0 + im] : 1.f;
                        s_w[im * kTgt32 + k] = wk;
                        weighted = weighted || wk != 0.f;
                    }
                    // offset of the target-group origin from the shifted chunk origin, as hi + lo
                    const double D0 = (to[0] - so[0]) - shk[0], D1 = (to[1] - so[1]) - shk[1],
                                 D2 = (to[2] - so[2]) - shk[2];
                    float* dl = s_delta + 6 * (im * kTgt32 + k);
                    dl[0] = (float)D0; dl[1] = (float)D1; dl[2] = (float)D2;
                    dl[3] = (float)(D0 - (double)dl[0]); dl[4] = (float)(D1 - (double)dl[1]);
                    dl[5] = (float)(D2 - (double)dl[2]);
                    const double reach = kNearFactor * (to[3] + so[3]);
                    if (D0 * D0 + D1 * D1 + D2 * D2 <= reach * reach) nr |= k < 2 ? kUnitNear0 : kUnitNear1;
                }
                if (kTrim) {
                    // the chunk's bounding sphere against the ball, with a margin: the exact
                    // per-source test decides everything near the sphere
                    const double c0 = so[0] + sh[0], c1 = so[1] + sh[1], c2 = so[2] + sh[2];
                    const double c2s = c0 * c0 + c1 * c1 + c2 * c2;
                    const double ro = a.Rb * (1.0 + 1e-12) + so[3], ri = a.Rb * (1.0 - 1e-12) - so[3];
                    if (c2s > ro * ro) nr = kUnitOutside;
                    else if (ri < 0.0 || c2s > ri * ri) nr |= kUnitStraddle;
                }
                if (!kGrad && !weighted) nr = kUnitOutside;   // padding image of every group: skip
                if (a.chunk_nimg && im >= a.chunk_nimg[chunk]) nr = kUnitOutside;   // past the chunk's list
                s_near[im] = nr;
            }
            const long long limit = a.inject ? (1LL << 12) : kCopySpinLimit;
            if (tid == 0 && !mbar_wait(&s_bar, phase, limit)) s_fail = 1;
            phase ^= 1u;
            __syncthreads();
            if (s_fail) {
                // the copy never completed: report it, give it one more bounded wait, leave
                if (tid == 0) {
                    for (int k = 0; k < a.n_status; ++k) atomicOr(a.status + k, kStatTimeout);
                    mbar_wait(&s_bar, phase ^ 1u, limit);
                }
                return;
            }
            cur_chunk = chunk;
        }
        const float* dl = s_delta + 6 * (img * kTgt32 * ncls);
        // the offsets of target group g's thread target (its class's entry) and the weights
        auto dptr = [&](int g) { return dl + 6 * (g * ncls + (kGrad ? 0 : s_tcls[g][tid])); };
        const int cls = s_near[img];
        if ((kTrim || !kGrad || a.chunk_nimg) && (cls & kUnitOutside)) {
            ++u;
            continue;
        }
        // potential only: the weight of each target group for this image (1, or +-1 and 0
        // for the two-layer check sums); multiplying by it is exact
        auto wpair = [&](int j) {
            const float* wl = s_w + img * kTgt32 * ncls;
            return make_float2(wl[2 * j * ncls + (kGrad ? 0 : s_tcls[2 * j][tid])],
                               wl[(2 * j + 1) * ncls + (kGrad ? 0 : s_tcls[2 * j + 1][tid])]);
        };
        // sources the unit's pair loops run over: the staged chunk, or for a unit that
        // straddles the ball its sources inside the ball, compacted (padded to whole blocks
        // of 4 with far-away zero charges)
        const float4* uhi = s_hi;
        const float4* ulo = s_lo;
        int un = kNearChunk;
        if (kTrim && (cls & kUnitStraddle)) {
            __syncthreads();                 // the previous unit is done with the compacted copy
            const double* sh = a.shifts + 3 * (Sp->shift0 + img);
            const double* xp = a.src_x + 3 * (chunk * kNearChunk + tid);
            const bool keep = in_ball(xp[0], xp[1], xp[2], sh, a.Rb);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int lane = tid & 31, warp = tid >> 5;
            if (lane == 0) s_wcnt[warp] = __popc(m);
            __syncthreads();
            int base = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kThreads32 / 32; ++w) {
                base += w < warp ? s_wcnt[w] : 0;
                total += s_wcnt[w];
            }
            const int pos = base + __popc(m & ((1u << lane) - 1u));
            if (keep) {
                s_hm[2 * pos] = s_hi[2 * tid];
                s_hm[2 * pos + 1] = s_hi[2 * tid + 1];
                s_hm[2 * kNearChunk + 2 * pos] = s_lo[2 * tid];
                s_hm[2 * kNearChunk + 2 * pos + 1] = s_lo[2 * tid + 1];
            }
            const int padded = (total + kNearFold - 1) / kNearFold * kNearFold;
            if (tid >= total && tid < padded) {
                s_hm[2 * tid] = make_float4(1.0e3f, 1.0e3f, 1.0e3f, 1.0e3f);
                s_hm[2 * tid + 1] = make_float4(1.0e3f, 1.0e3f, 0.f, 0.f);
                s_hm[2 * kNearChunk + 2 * tid] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_hm[2 * kNearChunk + 2 * tid + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            uhi = s_hm;
            ulo = s_hm + 2 * kNearChunk;
            un = padded;
        }
        const int n_pairs = pair1_live ? 2 : 1;
        if constexpr (kFF) {
            // every unit in float-float: t' = t + delta as hi + lo
#pragma unroll 1
            for (int j = 0; j < n_pairs; ++j) {
                const float* d0 = dptr(2 * j);
                const float* d1 = dptr(2 * j + 1);
                float2 nTh[3], nTl[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float2 e;
                    const float2 th = two_sum2(s_th[c][j][tid], make_float2(d0[c], d1[c]), e);
                    const float2 tl = __fadd2_rn(__fadd2_rn(s_tl[c][j][tid], make_float2(d0[3 + c], d1[3 + c])), e);
                    nTh[c] = neg2(th);
                    nTl[c] = neg2(tl);
                }
                float2 acc[4][2];
#pragma unroll
                for (int qi = 0; qi < 4; ++qi) acc[qi][0] = acc[qi][1] = make_float2(0.f, 0.f);
                const float tau2 = Sp->tau2;
                if (cls & (j ? kUnitNear1 : kUnitNear0))
                    pair_loop_ff<kGrad, true>(uhi, ulo, nTh, nTl, acc, tau2, un);
                else
                    pair_loop_ff<kGrad, false>(uhi, ulo, nTh, nTl, acc, tau2, un);
                if constexpr (!kGrad) {
                    acc[0][0] = __fmul2_rn(acc[0][0], wpair(j));
                    acc[0][1] = __fmul2_rn(acc[0][1], wpair(j));
                }
#pragma unroll
                for (int qi = 0; qi < NQ; ++qi) {
                    two_sum_acc2(s_acc[qi][j][0][tid], s_acc[qi][j][1][tid], acc[qi][0]);
                    s_acc[qi][j][1][tid] = __fadd2_rn(s_acc[qi][j][1][tid], acc[qi][1]);
                }
            }
        } else if (cls & kUnitNear) {
            // near pairs: t' = t + delta in float-float (hi by rounding, lo = exact remainder +
            // both lo parts); a pair whose two groups are both far takes the far loop alone
#pragma unroll 1
            for (int j = 0; j < n_pairs; ++j) {
                const float* d0 = dptr(2 * j);
                const float* d1 = dptr(2 * j + 1);
                if (!(cls & (j ? kUnitNear1 : kUnitNear0))) {
                    const float2 tx = s_th[0][j][tid], ty = s_th[1][j][tid], tz = s_th[2][j][tid];
                    const float2 nx[1] = {make_float2(-(tx.x + d0[0]), -(tx.y + d1[0]))};
                    const float2 ny[1] = {make_float2(-(ty.x + d0[1]), -(ty.y + d1[1]))};
                    const float2 nz[1] = {make_float2(-(tz.x + d0[2]), -(tz.y + d1[2]))};
                    float2 aphi[1] = {make_float2(0.f, 0.f)}, agx[1] = {aphi[0]}, agy[1] = {aphi[0]},
                           agz[1] = {aphi[0]};
                    pair_loop_far<kGrad, 1>(uhi, nx, ny, nz, aphi, agx, agy, agz, un);
                    if constexpr (!kGrad) aphi[0] = __fmul2_rn(aphi[0], wpair(j));
                    two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid], aphi[0]);
                    if (kGrad) {
                        two_sum_acc2(s_acc[1 % NQ][j][0][tid], s_acc[1 % NQ][j][1][tid], agx[0]);
                        two_sum_acc2(s_acc[2 % NQ][j][0][tid], s_acc[2 % NQ][j][1][tid], agy[0]);
                        two_sum_acc2(s_acc[3 % NQ][j][0][tid], s_acc[3 % NQ][j][1][tid], agz[0]);
                    }
                    continue;
                }
                // target lo parts are read from global memory: near pairs are rare
                const int64_t i0 = (cur_tile * kTgt32 + 2 * j) * kGroup + tid;
                const int64_t i1 = i0 + kGroup;
                const float4 C0 = a.tgt_lo[2 * i0], D0 = a.tgt_lo[2 * i0 + 1];
                const float4 C1 = a.tgt_lo[2 * i1], D1 = a.tgt_lo[2 * i1 + 1];
                const float2 tls[3] = {make_float2(C0.x, C1.x), make_float2(C0.z, C1.z), make_float2(D0.x, D1.x)};
                float2 nh[3], nl[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 th = s_th[c][j][tid], tl = tls[c];
                    float e0, e1;
                    const float h0 = two_sum(th.x, d0[c], e0);
                    const float h1 = two_sum(th.y, d1[c], e1);
                    nh[c] = make_float2(-h0, -h1);
                    nl[c] = make_float2(-(e0 + (tl.x + d0[3 + c])), -(e1 + (tl.y + d1[3 + c])));
                }
                float2 aphi = make_float2(0.f, 0.f), aphi_lo = aphi, agx = aphi, agy = aphi, agz = aphi;
                const float tau2 = Sp->tau2;
                pair_loop_near<kGrad>(uhi, ulo, nh[0], nh[1], nh[2], nl[0], nl[1], nl[2], aphi, aphi_lo, agx, agy,
                                      agz, tau2, un);
                if constexpr (!kGrad) {
                    aphi = __fmul2_rn(aphi, wpair(j));
                    aphi_lo = __fmul2_rn(aphi_lo, wpair(j));
                }
                two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid], aphi);
                s_acc[0][j][1][tid] = __fadd2_rn(s_acc[0][j][1][tid], aphi_lo);
                if (kGrad) {
                    two_sum_acc2(s_acc[1 % NQ][j][0][tid], s_acc[1 % NQ][j][1][tid], agx);
                    two_sum_acc2(s_acc[2 % NQ][j][0][tid], s_acc[2 % NQ][j][1][tid], agy);
                    two_sum_acc2(s_acc[3 % NQ][j][0][tid], s_acc[3 % NQ][j][1][tid], agz);
                }
            }
        } else if (!pair1_live) {
            // the first packed target pair alone
            const float* d0 = dptr(0);
            const float* d1 = dptr(1);
            const float2 tx = s_th[0][0][tid], ty = s_th[1][0][tid], tz = s_th[2][0][tid];
            const float2 nx[1] = {make_float2(-(tx.x + d0[0]), -(tx.y + d1[0]))};
            const float2 ny[1] = {make_float2(-(ty.x + d0[1]), -(ty.y + d1[1]))};
            const float2 nz[1] = {make_float2(-(tz.x + d0[2]), -(tz.y + d1[2]))};
            float2 aphi[1] = {make_float2(0.f, 0.f)}, agx[1] = {aphi[0]}, agy[1] = {aphi[0]}, agz[1] = {aphi[0]};
            pair_loop_far<kGrad, 1>(uhi, nx, ny, nz, aphi, agx, agy, agz, un);
            if constexpr (!kGrad) aphi[0] = __fmul2_rn(aphi[0], wpair(0));
            two_sum_acc2(s_acc[0][0][0][tid], s_acc[0][0][1][tid], aphi[0]);
            if (kGrad) {
                two_sum_acc2(s_acc[1 % NQ][0][0][tid], s_acc[1 % NQ][0][1][tid], agx[0]);
                two_sum_acc2(s_acc[2 % NQ][0][0][tid], s_acc[2 % NQ][0][1][tid], agy[0]);
                two_sum_acc2(s_acc[3 % NQ][0][0][tid], s_acc[3 % NQ][0][1][tid], agz[0]);
            }
        } else {
            float2 nx[2], ny[2], nz[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float* d0 = dptr(2 * j);
                const float* d1 = dptr(2 * j + 1);
                const float2 tx = s_th[0][j][tid], ty = s_th[1][j][tid], tz = s_th[2][j][tid];
                nx[j] = make_float2(-(tx.x + d0[0]), -(tx.y + d1[0]));
                ny[j] = make_float2(-(ty.x + d0[1]), -(ty.y + d1[1]));
                nz[j] = make_float2(-(tz.x + d0[2]), -(tz.y + d1[2]));
            }
            float2 aphi[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            float2 agx[2] = {aphi[0], aphi[0]}, agy[2] = {aphi[0], aphi[0]}, agz[2] = {aphi[0], aphi[0]};
            pair_loop_far<kGrad, 2>(uhi, nx, ny, nz, aphi, agx, agy, agz, un);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if constexpr (!kGrad) aphi[j] = __fmul2_rn(aphi[j], wpair(j));
                two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid], aphi[j]);
                if (kGrad) {
                    two_sum_acc2(s_acc[1 % NQ][j][0][tid], s_acc[1 % NQ][j][1][tid], agx[j]);
                    two_sum_acc2(s_acc[2 % NQ][j][0][tid], s_acc[2 % NQ][j][1][tid], agy[j]);
                    two_sum_acc2(s_acc[3 % NQ][j][0][tid], s_acc[3 % NQ][j][1][tid], agz[j]);
                }
            }
        }
        ++u;
    }
    if (cur_tile >= 0) flush(cur_tile, cur_first);
    }
}

// ---------------------------------------------------------------------------
// FP64 kernel
// ---------------------------------------------------------------------------
struct Near64Args {
    const double4_32a* src;      // (x, y, z, q), absolute
    const double4_32a* tgt;      // (x, y, z, -)
    const double* shifts;
    double* partial;             // [tiles][max_contrib][4 or 1][kTile64]
    double Rb;                   // > 0: keep a source image x + p only if |x + p| <= Rb (get step 2)
    int64_t U, W;                // units, work items
    int* counter;                // next work item
    int max_contrib;
    NearSysTable tab;
    // two-layer check sums (potential only): each target's class c (0..n_cls-1) rides in its
    // pack's fourth component; the image vector of (class c, image j) is
    // shifts[shift0 + c n_img + j], its weight img_w[shift0 + c n_img + j].  n_cls = 1 and a
    // null table: one image list, weight 1.
    const float* img_w;
    int n_cls;
};


template <bool kGrad>
__global__ void __launch_bounds__(kThreads64) k_near64(Near64Args a) {
    __shared__ double4_32a s_src[kNearChunk];
    __shared__ double4_32a s_srcm[kNearChunk];        // the chunk with the image's masked charges
    constexpr int NQ = kGrad ? 4 : 1;
    __shared__ int s_item;
    const int tid = threadIdx.x;
    int64_t item = 0;
    double tx = 0, ty = 0, tz = 0;
    int tcls = 0;                        // the target's class (two-layer check sums)
    double acc[NQ];

    auto flush = [&](int64_t tile, int64_t first_unit) {
        const int64_t slot = item - sk_owner(first_unit, a.U, a.W);
        double* dst = a.partial + ((tile * a.max_contrib + slot) * NQ) * kTile64;
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi) dst[qi * kTile64 + tid] = acc[qi];
    };

    for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    item = s_item;
    __syncthreads();                     // every thread has the item before s_item changes
    if (item >= a.W) break;
    int64_t u = sk_bound(item, a.U, a.W);
    const int64_t u_end = sk_bound(item + 1, a.U, a.W);
    int sb = near_sys_by_unit(a.tab, u);
    NearSys S = near_sys_get(a.tab, sb);
    int64_t cur_tile = -1, cur_chunk = -1, cur_first = 0;
    while (u < u_end) {
        while (u >= S.unit0 + near_sys_units(S)) S = near_sys_get(a.tab, ++sb);
        const int64_t upt = S.n_chunks * S.n_img;
        const int64_t local = u - S.unit0;
        const int64_t tile_l = local / upt;
        const int64_t rem = local - tile_l * upt;
        const int64_t chunk_l = rem / S.n_img;
        const int img = (int)(rem - chunk_l * S.n_img);
        const int64_t tile = S.tile0 + tile_l;
        const int64_t chunk = S.src_chunk0 + (chunk_l * S.chunk_stride) % S.n_chunks;
        if (tile != cur_tile) {
            if (cur_tile >= 0) flush(cur_tile, cur_first);
            const double4_32a t = a.tgt[tile * kTile64 + tid];
            tx = t.x; ty = t.y; tz = t.z;
            // a class outside 0..n_cls-1 reads class 0: the index stays inside the tables
            tcls = (!kGrad && a.n_cls > 1 && t.w >= 0.0 && t.w < (double)a.n_cls) ? (int)t.w : 0;
#pragma unroll
            for (int qi = 0; qi < NQ; ++qi) acc[qi] = 0.0;
            cur_tile = tile;
            cur_first = S.unit0 + tile_l * upt;
            cur_chunk = -1;
        }
        if (chunk != cur_chunk) {
            __syncthreads();
            for (int i = tid; i < kNearChunk; i += kThreads64) s_src[i] = a.src[chunk * kNearChunk + i];
            __syncthreads();
            cur_chunk = chunk;
        }
        // y - x_i - p with the shift folded into the target
        const double* sh = a.shifts + 3 * (S.shift0 + img);
        double w = 1.0;                  // the target's weight (potential only); exact in the fma
        if (!kGrad && a.img_w) {
            const int e = S.shift0 + tcls * S.n_img + img;
            sh = a.shifts + 3 * e;
            w = (double)a.img_w[e];
            if (a.n_cls == 1 && w == 0.0) {   // one image list: the unit's weight, uniform
                ++u;
                continue;
            }
        }
        const double px = tx - sh[0], py = ty - sh[1], pz = tz - sh[2];
        const double4_32a* src = s_src;
        if (a.Rb > 0.0) {
            __syncthreads();
            const double4_32a Q = s_src[tid];
            s_srcm[tid] = make_double4_32a(Q.x, Q.y, Q.z, in_ball(Q.x, Q.y, Q.z, sh, a.Rb) ? Q.w : 0.0);
            __syncthreads();
            src = s_srcm;
        }
#pragma unroll 4
        for (int s = 0; s < kNearChunk; ++s) {
            const double4_32a Q = src[s];
            const double ex = Q.x - px, ey = Q.y - py, ez = Q.z - pz;   // x_i + p - y
            const double r2 = fma(ez, ez, fma(ey, ey, ex * ex));
            const double ri = rsqrt_f64_k0(r2);           // K(0) = 0
            const double qr = Q.w * ri;
            if (kGrad)
                acc[0] += qr;
            else
                acc[0] = fma(w, qr, acc[0]);
            if (kGrad) {
                const double w = qr * ri * ri;
                acc[1 % NQ] = fma(ex, w, acc[1 % NQ]);
                acc[2 % NQ] = fma(ey, w, acc[2 % NQ]);
                acc[3 % NQ] = fma(ez, w, acc[3 % NQ]);
            }
        }
        ++u;
    }
    if (cur_tile >= 0) flush(cur_tile, cur_first);
    }
}

// ---------------------------------------------------------------------------
// Reduction of the partial slots (fixed order: slot 0, 1, ...) for packed target
// index i < n_valid (tile = i / tile_size is the partial-buffer row).
// ---------------------------------------------------------------------------
// A block sums the slots of 32 consecutive targets (one per lane) and one quantity: its 8
// warps take every 8th slot, and the 8 warp sums are added in a fixed order in shared
// memory, so the result does not depend on timing.  Tiles never mix within a block (the
// tile sizes are multiples of 32).

__global__ void __launch_bounds__(32 * kReduceWarps) k_near_reduce(const double* __restrict__ partial,
                                                                   int64_t n_valid, int tile_size, int nq,
                                                                   NearSysTable tab, int64_t U, int64_t W,
                                                                   int max_contrib, double* __restrict__ out_phi,
                                                                   double* __restrict__ out_grad) {
    __shared__ double s_part[kReduceWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int qi = blockIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int64_t i = i0 + lane;
    const int64_t tile = i0 / tile_size;
    const int loc = (int)(i - tile * tile_size);
    const NearSys S = near_sys_get(tab, near_sys_by_tile(tab, tile));
    const int64_t upt = S.n_chunks * S.n_img;
    const int64_t first = S.unit0 + (tile - S.tile0) * upt;
    const int n = (int)(sk_owner(first + upt - 1, U, W) - sk_owner(first, U, W) + 1);
    const double* src = partial + (tile * max_contrib * nq + qi) * (int64_t)tile_size + loc;
    const int64_t stride = (int64_t)nq * tile_size;
    double acc = 0.0;
    if (i < n_valid)
        for (int sl = warp; sl < n; sl += kReduceWarps) acc += src[sl * stride];
    s_part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && i < n_valid) {
        double v = s_part[0][lane];
#pragma unroll
        for (int w = 1; w < kReduceWarps; ++w) v += s_part[w][lane];
        if (qi == 0)
            out_phi[i] = v;
        else if (out_grad)
            out_grad[3 * i + qi - 1] = v;
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
// The instance of k_near32 a launch runs: trimmed near sets and float-float take the larger
// register budget, the others the variant's.
using Near32Kernel = void (*)(Near32Args);
Near32Kernel near32_instance(bool grad, int variant, bool trimmed, bool ff) {
    constexpr int B0 = kNear32MinBlocks[0], B1 = kNear32MinBlocks[1];
    if (ff) {
        if (trimmed) return grad ? k_near32<true, B0, true, true> : k_near32<false, B0, true, true>;
        return grad ? k_near32<true, B0, false, true> : k_near32<false, B0, false, true>;
    }
    if (trimmed) return grad ? k_near32<true, B0, true, false> : k_near32<false, B0, true, false>;
    if (variant == 1) return grad ? k_near32<true, B1, false, false> : k_near32<false, B1, false, false>;
    return grad ? k_near32<true, B0, false, false> : k_near32<false, B0, false, false>;
}

// Dynamic shared memory beyond what needs no opt-in (a ball that keeps many images, with
// their offsets per target group): raise the instance's limit to what the launch asks for.
cudaError_t near32_allow_smem(Near32Kernel kernel, size_t smem) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes + smem <= (size_t)48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

size_t near32_dyn_smem(int n_img, bool trimmed, bool grad, int n_cls) {
    const size_t head = ((6 * kTgt32 * (size_t)n_cls * n_img + n_img + (grad ? 0 : kTgt32 * (size_t)n_cls * n_img) +
                          3) / 4) * sizeof(float4);
    return head + (trimmed ? sizeof(float4) * 4 * kNearChunk : 0);   // compacted sources (hi, lo parts)
}

cudaError_t launch_near32(bool grad, const float4* src_hi, const float4* src_lo, const double* src_org,
                          const float4* tgt_hi, const float4* tgt_lo, const double* tgt_org, const double* shifts,
                          double* partial, const NearPlanLaunch& L, cudaStream_t st, int variant,
                          const double* src_x, double Rb, bool ff, const int* grp_cls, const float* img_w,
                          int n_cls, const double* grp_sub, const int* chunk_img0, const int* chunk_nimg) {
    Near32Args a;
    a.chunk_img0 = chunk_img0;
    a.chunk_nimg = chunk_nimg;
    if ((chunk_img0 != nullptr) != (chunk_nimg != nullptr) || (chunk_img0 && (n_cls > 1 || Rb > 0.0)))
        return cudaErrorInvalidValue;
    a.status = L.status;
    a.n_status = L.n_status;
    a.inject = L.inject;
    if (!L.status || L.n_status < 1) return cudaErrorInvalidValue;
    a.src_hi = src_hi; a.src_lo = src_lo; a.src_org = src_org;
    a.tgt_hi = tgt_hi; a.tgt_lo = tgt_lo; a.tgt_org = tgt_org; a.shifts = shifts;
    a.partial = partial; a.U = L.U; a.W = L.W; a.counter = L.counter; a.max_contrib = L.max_contrib;
    a.max_img = L.max_img;
    a.tab = L.tab;
    {
        // the partial buffer as the debug bounds checks see it (a test may shrink it)
        const int64_t real = L.n_tiles * L.max_contrib * (grad ? 4 : 1) * kTile32;
        a.limit = L.debug_limit > 0 && L.debug_limit < real ? L.debug_limit : real;
    }
    a.src_x = src_x;
    a.Rb = Rb;
    if (n_cls < 1 || (n_cls > 1 && (!grp_cls || !grp_sub || !img_w || grad || Rb > 0.0)) || (img_w && grad))
        return cudaErrorInvalidValue;
    a.grp_cls = grp_cls;
    a.grp_sub = grp_sub;
    a.img_w = img_w;
    a.n_cls = n_cls;
    const size_t smem = near32_dyn_smem(L.max_img, Rb > 0.0, grad, n_cls);
    if (!L.counter) return cudaErrorInvalidValue;
    const cudaError_t e = cudaMemsetAsync(L.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const unsigned G = (unsigned)L.G;
    const auto kernel = near32_instance(grad, variant, Rb > 0.0, ff);
    const cudaError_t ea = near32_allow_smem(kernel, smem);
    if (ea != cudaSuccess) return ea;
    kernel<<<G, kThreads32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_near64(bool grad, const double4_32a* src, const double4_32a* tgt, const double* shifts,
                          double* partial, const NearPlanLaunch& L, cudaStream_t st, double Rb, const float* img_w,
                          int n_cls) {
    if (n_cls < 1 || (n_cls > 1 && !img_w) || (img_w && (grad || Rb > 0.0))) return cudaErrorInvalidValue;
    Near64Args a;
    a.src = src; a.tgt = tgt; a.shifts = shifts; a.partial = partial; a.Rb = Rb;
    a.img_w = img_w; a.n_cls = n_cls;
    a.U = L.U; a.W = L.W; a.counter = L.counter; a.max_contrib = L.max_contrib; a.tab = L.tab;
    if (!L.counter) return cudaErrorInvalidValue;
    const cudaError_t e = cudaMemsetAsync(L.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (grad)
        k_near64<true><<<(unsigned)L.G, kThreads64, 0, st>>>(a);
    else
        k_near64<false><<<(unsigned)L.G, kThreads64, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_near_reduce(const double* partial, int64_t n_valid, int tile_size, int nq,
                               const NearPlanLaunch& L, double* out_phi, double* out_grad, cudaStream_t st) {
    if (n_valid <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((n_valid + 31) / 32), (unsigned)nq);
    k_near_reduce<<<grid, 32 * kReduceWarps, 0, st>>>(partial, n_valid, tile_size, nq, L.tab, L.U, L.W, L.max_contrib, out_phi,
                                     out_grad);
    return cudaGetLastError();
}

int near32_occupancy_ctas(int n_img, int variant, bool trimmed, bool ff, bool grad, int n_cls) {
    int nb = 0;
    const size_t smem = near32_dyn_smem(n_img, trimmed, grad, n_cls);
    const Near32Kernel kernel = near32_instance(grad, variant, trimmed, ff);
    if (near32_allow_smem(kernel, smem) == cudaSuccess)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads32, smem);
    return nb < 1 ? 1 : nb;
}

int near64_occupancy_ctas() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_near64<true>, kThreads64, 0);
    return nb < 1 ? 1 : nb;
}

}  // namespace psum
