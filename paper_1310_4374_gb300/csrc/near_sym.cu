// Symmetric near-field kernels for the charge sums (targets = sources): each pair of
// tiles is taken once with every image of the block, and a pair (i, j, p) and its mirror
// (j, i, -p) share one offset and one 1/r -- k_near32s (FP32C and float-float) and
// k_near64s (FP64), their fixed-order reduction and launchers.  The one-sided kernels and
// the shared helpers are in near.cu and near_common.cuh.
#include "near_common.cuh"

namespace psum {

// ---------------------------------------------------------------------------
// Symmetric charge kernel (FP32C and float-float, potential and field at the charges,
// block image sets, one or many systems).
// With the charges as both targets and sources, the pair (i, j, p) and its mirror
// (j, i, -p) are one distance apart: one offset, one rsqrt and one 1/r^2 serve the
// target's sum (the action, q_j / r) and the source's (the reaction, q_i / r, field
// with the opposite sign).  The image set {p} of a block is symmetric, so the pairs
// of tiles (a, b), a < b, each taken once with every image, cover the whole sum.  A tile
// against itself (a = b) takes one image of each mirror pair {p, -p}, p != 0 (the one whose
// first nonzero coordinate is positive), with reactions onto its own charges, and the zero
// image by the one-sided pair loops (near_common.cuh), K(0) = 0.
//
//   * the work item is (tile pair (a, b), group of images); items are taken from a
//     device counter; the action on tile a goes to partial slot (a, b, g), the reaction
//     on tile b to slot (b, a, g), so every slot has one writer and the reduction adds
//     a tile's n_tiles * n_g slots in a fixed order;
//   * per source chunk of tile b and image, a warp's 32 lanes (4 targets each) visit the
//     chunk in 2 rounds of 32 source pairs (the chunk re-laid in shared memory as pairs,
//     (x0,x1,y0,y1),(z0,z1,q0,q1), so that one packed operation serves both sources of
//     a pair for one target; round g pairs source 64 g + l with 64 g + l + 32, so each
//     half of a packed sum takes a run of consecutive sources of the spatial order): at
//     step k lane l takes pair (l + k) mod 32 of the round and
//     adds its targets' terms to the pair's reaction sums, which then move one lane down
//     (shuffles), so after 32 steps lane l holds the reactions of pair l over the warp's
//     128 targets; the 4 warps keep private compensated (hi, lo) sums per source,
//     combined in a fixed order when the chunk is done (near units keep one source per
//     step in the original layout);
//   * near pairs (as in the one-sided units) take float-float offsets, K(0) = 0 and
//     blocks of 4 terms with compensated sums, on both sides;
//   * kFF: every pair in float-float arithmetic (the one-sided float-float loop's offsets,
//     r^2 and 1/r, shared), one packed target pair per rotation pass.
// Work items of several systems (batches) follow one another; a system's table entry
// gives its first item, tiles, chunks, images and partial block.
// ---------------------------------------------------------------------------
struct Near32SymArgs {
    const float4* pk_hi;     // the charges' pack: 2 float4 per point, (x,x,y,y),(z,z,q,q) offsets
    const float4* pk_lo;     // their float32 rounding remainders
    const double* org;       // 4 per group of 128 points: origin x, y, z and radius
    const float4* ext;       // per group: bounding-box half extents about the origin (nullptr: the
                             // near test compares origin distances with the radii alone)
    const double* shifts;    // image vectors, 3 per image, systems one after another
    double* partial;         // per system [n_tiles][n_tiles * n_g][4][kTile32] from part0
    SymSysTable tab;
    int64_t W;               // work items of all systems
    int max_ipg;             // largest images per group (shared-memory layout)
    int* counter;
    int* status;
    int n_status;
    int inject;              // test hook: expect 16 bytes more than the copies bring
    int64_t limit;           // doubles of the partial buffer (debug bounds checks)
};

// compensated float32 (hi, lo) += v
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    float e;
    hi = two_sum(hi, v, e);
    lo += e;
}

// One far step over a pair of sources (s0, s1) in the pair layout A = (x0, x1, y0, y1),
// B = (z0, z1, q0, q1): the lane's 4 targets (duplicated coordinates, negated offsets) each
// take both sources in one packed operation; the action sums keep the two sources in their
// two halves (folded once per unit), the reaction sums keep the two sources apart, so no
// per-step fold is needed.
__device__ __forceinline__ void sym_far_step_pair(float4 A, float4 B, const float2 (&nx)[4], const float2 (&ny)[4],
                                                  const float2 (&nz)[4], const float2 (&tq)[4], float2 (&aphi)[4],
                                                  float2 (&agx)[4], float2 (&agy)[4], float2 (&agz)[4],
                                                  float2& rp, float2& rx, float2& ry, float2& rz) {
    const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w), sz = make_float2(B.x, B.y);
    const float2 sq = make_float2(B.z, B.w);
    float2 bp;                 // the 4 targets' potential reactions, summed before the running sum
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 ex = __fadd2_rn(sx, nx[i]);
        const float2 ey = __fadd2_rn(sy, ny[i]);
        const float2 ez = __fadd2_rn(sz, nz[i]);
        float2 r2 = __fmul2_rn(ex, ex);
        r2 = __ffma2_rn(ey, ey, r2);
        r2 = __ffma2_rn(ez, ez, r2);
        const float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        const float2 ri2 = __fmul2_rn(ri, ri);
        const float2 qa = __fmul2_rn(sq, ri);
        aphi[i] = __fadd2_rn(aphi[i], qa);
        const float2 wa = __fmul2_rn(qa, ri2);
        agx[i] = __ffma2_rn(ex, wa, agx[i]);
        agy[i] = __ffma2_rn(ey, wa, agy[i]);
        agz[i] = __ffma2_rn(ez, wa, agz[i]);
        const float2 qb = __fmul2_rn(tq[i], ri);
        bp = i == 0 ? qb : __fadd2_rn(bp, qb);
        const float2 wb = __fmul2_rn(qb, ri2);
        rx = __ffma2_rn(ex, wb, rx);
        ry = __ffma2_rn(ey, wb, ry);
        rz = __ffma2_rn(ez, wb, rz);
    }
    rp = __fadd2_rn(rp, bp);
}

// The same far step with refined potential terms (PSUM_TERMS_REFINED).  The float32 term q/r
// carries the rounding of its offsets, of r^2, of the MUFU estimate z (0.58 ulp rms, measured)
// and of the product q z -- about one ulp of the term in all; on systems whose potential
// cancels strongly (tight dipoles: a potential of rms ~100 from terms whose root-sum-square is
// ~20x larger) these errors, not the sums, set the potential's accuracy.  Here:
//   * the offset e = s + n' is carried as eh + el: el = (s - (eh - n')) is the exact rounding
//     error of the sum wherever |n'| >= |s| component by component (Fast2Sum; where not, both
//     are small and so is the error left), and the target offset's own rounding enters r^2
//     through the per-target constant c0 = n' . n'_lo (n'_lo = -(t + D) - n', float64 unit
//     offset D), so r^2 = rh + 2 c with c = c0 + eh . el;
//   * 1/r is the pair z + k, with k the Newton correction -z (r^2 z^2 - 1) / 2 computed from that
//     r^2, and both products go into fused multiply-adds unrounded: the action adds q_s z to its
//     running sum and q_s k to a separate correction sum; the reaction forms the 4 targets'
//     corrections first and adds their q_t z on top.
// The field keeps the unrefined weight q z^3 (a few ulps of terms that cancel far less).  Per
// term about 0.41 ulp rms instead of 0.99 (float32 emulation of this arithmetic); per target
// and source pair 30 packed operations instead of 19 (the correction's -1/2 rides on the
// targets' charges for the reaction and on the action's correction sum).
__device__ __forceinline__ void sym_far_step_pair_refined(float4 A, float4 B, const float2 (&nx)[4],
                                                          const float2 (&ny)[4], const float2 (&nz)[4],
                                                          const float2 (&c0)[4], const float2 (&tq)[4],
                                                          const float2 (&tqh)[4],
                                                          float2 (&aphi)[4], float2 (&acor)[4], float2 (&agx)[4],
                                                          float2 (&agy)[4], float2 (&agz)[4], float2& rp, float2& rx,
                                                          float2& ry, float2& rz) {
    const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w), sz = make_float2(B.x, B.y);
    const float2 sq = make_float2(B.z, B.w);
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 z[4], k[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 ex = __fadd2_rn(sx, nx[i]);
        const float2 ey = __fadd2_rn(sy, ny[i]);
        const float2 ez = __fadd2_rn(sz, nz[i]);
        const float2 lx = __ffma2_rn(m1, __ffma2_rn(m1, nx[i], ex), sx);    // s - (e - n')
        const float2 ly = __ffma2_rn(m1, __ffma2_rn(m1, ny[i], ey), sy);
        const float2 lz = __ffma2_rn(m1, __ffma2_rn(m1, nz[i], ez), sz);
        float2 r2 = __fmul2_rn(ex, ex);
        r2 = __ffma2_rn(ey, ey, r2);
        r2 = __ffma2_rn(ez, ez, r2);
        float2 c = __ffma2_rn(ex, lx, c0[i]);
        c = __ffma2_rn(ey, ly, c);
        c = __ffma2_rn(ez, lz, c);
        z[i] = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        const float2 zz = __fmul2_rn(z[i], z[i]);
        const float2 rt = __ffma2_rn(make_float2(2.f, 2.f), c, r2);           // r^2 with its low part
        const float2 g = __ffma2_rn(rt, zz, m1);                               // r^2 z^2 - 1
        k[i] = __fmul2_rn(z[i], g);            // -2x the correction: the -1/2 goes into acor's scale and tqh
        const float2 ri3 = __fmul2_rn(z[i], zz);
        aphi[i] = __ffma2_rn(sq, z[i], aphi[i]);
        acor[i] = __ffma2_rn(sq, k[i], acor[i]);
        const float2 wa = __fmul2_rn(sq, ri3);
        agx[i] = __ffma2_rn(ex, wa, agx[i]);
        agy[i] = __ffma2_rn(ey, wa, agy[i]);
        agz[i] = __ffma2_rn(ez, wa, agz[i]);
        const float2 wb = __fmul2_rn(tq[i], ri3);
        rx = __ffma2_rn(ex, wb, rx);
        ry = __ffma2_rn(ey, wb, ry);
        rz = __ffma2_rn(ez, wb, rz);
    }
    float2 bp = __fmul2_rn(tqh[0], k[0]);
#pragma unroll
    for (int i = 1; i < 4; ++i) bp = __ffma2_rn(tqh[i], k[i], bp);
#pragma unroll
    for (int i = 0; i < 4; ++i) bp = __ffma2_rn(tq[i], z[i], bp);
    rp = __fadd2_rn(rp, bp);
}

// One near step: float-float offsets (hi + lo of both sides), K(0) = 0; the action's
// potential terms go to blk (a block of 4 steps), the reaction's potential (a block of
// the 4 targets' terms) into the compensated (rp, rpl).
__device__ __forceinline__ void sym_near_step(const float4* __restrict__ s_hi, const float4* __restrict__ s_lo,
                                              int si, const float2 (&nh)[2][3], const float2 (&nl)[2][3],
                                              const float2 (&tq)[2], float tau2, float2 (&blk)[2], bool first,
                                              float2 (&agx)[2], float2 (&agy)[2], float2 (&agz)[2], float& rp,
                                              float& rpl, float& rx, float& ry, float& rz) {
    const float4 A = s_hi[2 * si], B = s_hi[2 * si + 1];
    const float4 C = s_lo[2 * si], D = s_lo[2 * si + 1];
    const float2 sq = make_float2(B.z, B.w);
    float2 bp, bx, by, bz;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float2 ex = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), nh[j][0]), __fadd2_rn(make_float2(C.x, C.y), nl[j][0]));
        const float2 ey = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), nh[j][1]), __fadd2_rn(make_float2(C.z, C.w), nl[j][1]));
        const float2 ez = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), nh[j][2]), __fadd2_rn(make_float2(D.x, D.y), nl[j][2]));
        float2 r2 = __fmul2_rn(ex, ex);
        r2 = __ffma2_rn(ey, ey, r2);
        r2 = __ffma2_rn(ez, ez, r2);
        float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        ri.x = r2.x > tau2 ? ri.x : 0.f;                  // K(0) = 0 (Eq. 1), coincident_r2
        ri.y = r2.y > tau2 ? ri.y : 0.f;
        const float2 ri2 = __fmul2_rn(ri, ri);
        const float2 qa = __fmul2_rn(sq, ri);
        blk[j] = first ? qa : __fadd2_rn(blk[j], qa);
        const float2 wa = __fmul2_rn(qa, ri2);
        agx[j] = __ffma2_rn(ex, wa, agx[j]);
        agy[j] = __ffma2_rn(ey, wa, agy[j]);
        agz[j] = __ffma2_rn(ez, wa, agz[j]);
        const float2 qb = __fmul2_rn(tq[j], ri);
        const float2 wb = __fmul2_rn(qb, ri2);
        if (j == 0) {
            bp = qb;
            bx = __fmul2_rn(ex, wb);
            by = __fmul2_rn(ey, wb);
            bz = __fmul2_rn(ez, wb);
        } else {
            bp = __fadd2_rn(bp, qb);
            bx = __ffma2_rn(ex, wb, bx);
            by = __ffma2_rn(ey, wb, by);
            bz = __ffma2_rn(ez, wb, bz);
        }
    }
    two_sum_acc(rp, rpl, bp.x + bp.y);
    rx += bx.x + bx.y;
    ry += by.x + by.y;
    rz += bz.x + bz.y;
}

// One float-float step: the lane's packed target pair (negated offsets nTh + nTl, charges
// tqh + tql) against source si, both directions in float-float arithmetic (the one-sided
// loop's offsets, r^2 and Newton-refined 1/r, computed once).  The action goes to acc
// (hi, lo per quantity); the reaction, summed over the 2 targets, to the compensated scalar
// sums r[q] = (hi, lo).  kRenorm: near units (ff_renorm).
template <bool kRenorm>
__device__ __forceinline__ void sym_ff_step(const float4* __restrict__ s_hi, const float4* __restrict__ s_lo,
                                            int si, const float2 (&nTh)[3], const float2 (&nTl)[3], float2 tqh,
                                            float2 tql, float tau2, float2 (&acc)[4][2], float (&r)[4][2]) {
    const float4 A = s_hi[2 * si], B = s_hi[2 * si + 1], C = s_lo[2 * si], D = s_lo[2 * si + 1];
    const float2 sh[3] = {make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(B.x, B.y)};
    const float2 sl[3] = {make_float2(C.x, C.y), make_float2(C.z, C.w), make_float2(D.x, D.y)};
    const float2 qh = make_float2(B.z, B.w), ql = make_float2(D.z, D.w);
    float2 eh[3], el[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 err;
        eh[c] = two_sum2(sh[c], nTh[c], err);
        el[c] = __fadd2_rn(__fadd2_rn(sl[c], nTl[c]), err);
    }
    ff_renorm<kRenorm>(eh, el);
    const float2 p0 = __fmul2_rn(eh[0], eh[0]), p1 = __fmul2_rn(eh[1], eh[1]), p2 = __fmul2_rn(eh[2], eh[2]);
    float2 lo = __ffma2_rn(eh[0], eh[0], neg2(p0));
    lo = __fadd2_rn(lo, __ffma2_rn(eh[1], eh[1], neg2(p1)));
    lo = __fadd2_rn(lo, __ffma2_rn(eh[2], eh[2], neg2(p2)));
    float2 cr = __fmul2_rn(eh[0], el[0]);
    cr = __ffma2_rn(eh[1], el[1], cr);
    cr = __ffma2_rn(eh[2], el[2], cr);
    lo = __ffma2_rn(make_float2(2.f, 2.f), cr, lo);
    float2 e1, e2;
    const float2 s1 = two_sum2(p0, p1, e1);
    const float2 r2h = two_sum2(s1, p2, e2);
    const float2 r2l = __fadd2_rn(lo, __fadd2_rn(e1, e2));
    const float2 y = make_float2(rsqrt_mufu(r2h.x), rsqrt_mufu(r2h.y));
    const float2 ah = __fmul2_rn(r2h, y);
    const float2 ae = __ffma2_rn(r2h, y, neg2(ah));
    const float2 bh = __fmul2_rn(ah, y);
    const float2 be = __ffma2_rn(ah, y, neg2(bh));
    float2 h = __fadd2_rn(bh, make_float2(-1.f, -1.f));
    h = __fadd2_rn(h, be);
    h = __ffma2_rn(ae, y, h);
    h = __ffma2_rn(__fmul2_rn(r2l, y), y, h);
    float2 rih = y;
    float2 ril = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), y), h);
    if (!(r2h.x > tau2)) rih.x = ril.x = 0.f;             // K(0) = 0 (Eq. 1), coincident_r2
    if (!(r2h.y > tau2)) rih.y = ril.y = 0.f;
    float2 r2il;
    const float2 r2ih = ff_mul2(rih, ril, rih, ril, r2il);
    // action: q_s / r and q_s (s - t') / r^3
    float2 Pl;
    const float2 Ph = ff_mul2(qh, ql, rih, ril, Pl);
    ff_acc2(acc[0][0], acc[0][1], Ph, Pl);
    float2 wl;
    const float2 wh = ff_mul2(Ph, Pl, r2ih, r2il, wl);
    // reaction: q_t / r and q_t (s - t') / r^3, the 2 targets' terms added in float-float
    float2 Rl;
    const float2 Rh = ff_mul2(tqh, tql, rih, ril, Rl);
    float2 vl;
    const float2 vh = ff_mul2(Rh, Rl, r2ih, r2il, vl);
    float e;
    float t = two_sum(Rh.x, Rh.y, e);
    float u = (Rl.x + Rl.y) + e;
    r[0][0] = two_sum(r[0][0], t, e);
    r[0][1] += u + e;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 gl;
        const float2 gh = ff_mul2(wh, wl, eh[c], el[c], gl);
        ff_acc2(acc[1 + c][0], acc[1 + c][1], gh, gl);
        float2 kl;
        const float2 kh = ff_mul2(vh, vl, eh[c], el[c], kl);
        t = two_sum(kh.x, kh.y, e);
        u = (kl.x + kl.y) + e;
        r[1 + c][0] = two_sum(r[1 + c][0], t, e);
        r[1 + c][1] += u + e;
    }
}

template <int kMinB, bool kFF, bool kRefine = false>
__global__ void __launch_bounds__(kThreads32, kMinB) k_near32s(Near32SymArgs a) {
    static_assert(!(kFF && kRefine), "float-float pairs need no refinement");
    constexpr int kWarps = kThreads32 / 32;
    __shared__ float4 s_hi[2 * kNearChunk];
    __shared__ float4 s_lo[2 * kNearChunk];
    __shared__ float2 s_th[3][2][kThreads32];             // target offsets of tile a, [coord][pair]
    __shared__ float2 s_tq[2][kThreads32];                // target charges, [pair]
    __shared__ float2 s_tl[kFF ? 3 : 1][2][kThreads32];   // FF: target lo offsets
    __shared__ float2 s_tql[kFF ? 2 : 1][kThreads32];     // FF: target charge lo parts
    __shared__ float2 s_acc[4][2][2][kThreads32];         // action sums [quantity][pair][hi, lo]
    __shared__ float4 s_sp[kFF ? 1 : kNearChunk];         // the chunk as source pairs (x0,x1,y0,y1),(z0,z1,q0,q1)
    extern __shared__ float4 s_dyn4[];
    // reaction sums [warp][quantity][hi, lo][source], then [img_per_g][kTgt32][6] deltas and
    // [img_per_g] unit classes
    auto s_re = reinterpret_cast<float (*)[4][2][kNearChunk]>(s_dyn4);
    float* s_delta = (float*)s_dyn4 + kWarps * 4 * 2 * kNearChunk;
    int* s_near = (int*)(s_delta + 6 * kTgt32 * a.max_ipg);
    __shared__ int s_item;
    __shared__ int s_fail;
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int up = (lane + 1) & 31;
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        s_fail = 0;
    }
    __syncthreads();

    for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t item = s_item;
    __syncthreads();                     // every thread has the item before s_item changes
    if (item >= a.W) break;
    const SymSys S = a.tab.many ? a.tab.many[sym_sys_by_item(a.tab, item)] : a.tab.one;
    const int64_t local = item - S.item0;
    const int64_t pair = local / S.n_g;
    const int gi = (int)(local - pair * S.n_g);
    int64_t ta, tb;                      // the band's pair: ta <= tb (tiles of the system)
    sym_band_pair(S, pair, ta, tb);
    const bool diag = ta == tb;
    const int64_t TA = S.tile0 + ta;     // global tiles
    const int im0 = gi * S.img_per_g;
    const int nimg = min(S.img_per_g, S.n_img - im0);
    // targets of tile ta; zero the action sums
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int64_t i0 = (TA * kTgt32 + 2 * j) * kGroup + tid;
        const int64_t i1 = i0 + kGroup;
        const float4 A0 = a.pk_hi[2 * i0], B0 = a.pk_hi[2 * i0 + 1];
        const float4 A1 = a.pk_hi[2 * i1], B1 = a.pk_hi[2 * i1 + 1];
        s_th[0][j][tid] = make_float2(A0.x, A1.x);
        s_th[1][j][tid] = make_float2(A0.z, A1.z);
        s_th[2][j][tid] = make_float2(B0.x, B1.x);
        s_tq[j][tid] = make_float2(B0.z, B1.z);
        if (kFF) {
            const float4 C0 = a.pk_lo[2 * i0], D0 = a.pk_lo[2 * i0 + 1];
            const float4 C1 = a.pk_lo[2 * i1], D1 = a.pk_lo[2 * i1 + 1];
            s_tl[0][j][tid] = make_float2(C0.x, C1.x);
            s_tl[kFF ? 1 : 0][j][tid] = make_float2(C0.z, C1.z);
            s_tl[kFF ? 2 : 0][j][tid] = make_float2(D0.x, D1.x);
            s_tql[kFF ? j : 0][tid] = make_float2(D0.z, D1.z);
        }
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) s_acc[qi][j][0][tid] = s_acc[qi][j][1][tid] = make_float2(0.f, 0.f);
    }
    // the source chunks of tile tb (global group indices)
    const int64_t c0 = (S.tile0 + tb) * kTgt32;
    const int64_t c1 = c0 + (tb * kTgt32 + kTgt32 < S.n_chunks ? kTgt32 : S.n_chunks - tb * kTgt32);
    for (int64_t chunk = c0; chunk < c1; ++chunk) {
        __syncthreads();   // every thread is done with the previous chunk, deltas, classes and reactions
        // this warp's reaction sums for the chunk start at zero (private to the warp until the
        // combination below)
#pragma unroll
        for (int qi = 0; qi < 4; ++qi)
#pragma unroll
            for (int k = 0; k < kNearChunk / 32; ++k) s_re[warp][qi][0][32 * k + lane] = s_re[warp][qi][1][32 * k + lane] = 0.f;
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_expect_tx(&s_bar, 2 * kChunkBytes + (a.inject ? 16 : 0));
            bulk_g2s(s_hi, a.pk_hi + chunk * (2 * kNearChunk), kChunkBytes, &s_bar);
            bulk_g2s(s_lo, a.pk_lo + chunk * (2 * kNearChunk), kChunkBytes, &s_bar);
        }
        // the system's last chunk holds last_n charges and padding: source blocks of padding
        // alone are skipped (their reactions stay zero)
        const int nv = chunk == S.tile0 * kTgt32 + S.n_chunks - 1 && S.last_n > 0 ? S.last_n : kNearChunk;
        const int nb32 = (nv + 31) >> 5, nb64 = (nv + 63) >> 6;
        const double* so = a.org + 4 * chunk;
        for (int im = tid; im < nimg; im += kThreads32) {
            const double* sh = a.shifts + 3 * (S.shift0 + im0 + im);
            int nr = 0;
            if (diag) {
                const int sg = shift_sign(sh);
                if (sg < 0) {
                    s_near[im] = kUnitMirrored;
                    continue;
                }
                if (sg == 0) nr = kUnitSelf;
            }
            for (int k = 0; k < kTgt32; ++k) {
                const double* to = a.org + 4 * (TA * kTgt32 + k);
                const double D0 = (to[0] - so[0]) - sh[0], D1 = (to[1] - so[1]) - sh[1], D2 = (to[2] - so[2]) - sh[2];
                float* dl = s_delta + 6 * (im * kTgt32 + k);
                dl[0] = (float)D0; dl[1] = (float)D1; dl[2] = (float)D2;
                dl[3] = (float)(D0 - (double)dl[0]); dl[4] = (float)(D1 - (double)dl[1]);
                dl[5] = (float)(D2 - (double)dl[2]);
                bool near;
                if (a.ext) {
                    // the gap between the two bounding boxes bounds every pair distance from below
                    const float4 ht = a.ext[TA * kTgt32 + k], hs = a.ext[chunk];
                    const double g0 = fmax(0.0, fabs(D0) - ((double)ht.x + (double)hs.x));
                    const double g1 = fmax(0.0, fabs(D1) - ((double)ht.y + (double)hs.y));
                    const double g2 = fmax(0.0, fabs(D2) - ((double)ht.z + (double)hs.z));
                    const double gap = (kNearFactor - 1.0) * (to[3] + so[3]);
                    near = g0 * g0 + g1 * g1 + g2 * g2 <= gap * gap;
                } else {
                    const double reach = kNearFactor * (to[3] + so[3]);
                    near = D0 * D0 + D1 * D1 + D2 * D2 <= reach * reach;
                }
                if (near) nr |= k < 2 ? kUnitNear0 : kUnitNear1;
            }
            s_near[im] = nr;
        }
        const long long limit = a.inject ? (1LL << 12) : kCopySpinLimit;
        if (tid == 0 && !mbar_wait(&s_bar, phase, limit)) s_fail = 1;
        phase ^= 1u;
        __syncthreads();
        if (s_fail) {
            if (tid == 0) {
                for (int k = 0; k < a.n_status; ++k) atomicOr(a.status + k, kStatTimeout);
                mbar_wait(&s_bar, phase ^ 1u, limit);
            }
            return;
        }
        if (!kFF) {
            // the chunk again as source pairs for the far rotation: pair P = 32 g + l holds
            // sources 64 g + l and 64 g + l + 32, so that each half of a packed sum runs over
            // 32 consecutive sources of the spatial order (consecutive points of a lattice or
            // of dipoles alternate in sign: even and odd ones apart would each sum one sign)
            const int P = tid >> 1, h = tid & 1;
            const int sa = 64 * (P >> 5) + (P & 31);
            const float4 U = s_hi[2 * sa + h], V = s_hi[2 * (sa + 32) + h];
            s_sp[tid] = make_float4(U.x, V.x, U.z, V.z);
            __syncthreads();
        }
        for (int im = 0; im < nimg; ++im) {
            const float* dl = s_delta + 6 * (im * kTgt32);
            const int cls = s_near[im];
            if (cls & kUnitMirrored) continue;
            if constexpr (kFF) {
                // every unit in float-float: t' = t + delta as hi + lo, one packed pair at a time
#pragma unroll 1
                for (int j = 0; j < 2; ++j) {
                    const float* d0 = dl + 6 * (2 * j);
                    const float* d1 = dl + 6 * (2 * j + 1);
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
                    const float tau2 = S.tau2;
                    const bool nearj = cls & (j ? kUnitNear1 : kUnitNear0);
                    if (cls & kUnitSelf) {
                        if (nearj)
                            pair_loop_ff<true, true>(s_hi, s_lo, nTh, nTl, acc, tau2);
                        else
                            pair_loop_ff<true, false>(s_hi, s_lo, nTh, nTl, acc, tau2);
                    } else {
                        const float2 tqh = s_tq[j][tid], tql = s_tql[kFF ? j : 0][tid];
#pragma unroll 1
                        for (int g = 0; g < nb32; ++g) {
                            float r[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
                            for (int k = 0; k < 32; ++k) {
                                const int si = 32 * g + ((lane + k) & 31);
                                if (nearj)
                                    sym_ff_step<true>(s_hi, s_lo, si, nTh, nTl, tqh, tql, tau2, acc, r);
                                else
                                    sym_ff_step<false>(s_hi, s_lo, si, nTh, nTl, tqh, tql, tau2, acc, r);
#pragma unroll
                                for (int qi = 0; qi < 4; ++qi) {
                                    r[qi][0] = __shfl_sync(0xffffffffu, r[qi][0], up);
                                    r[qi][1] = __shfl_sync(0xffffffffu, r[qi][1], up);
                                }
                            }
                            const int s = 32 * g + lane;
#pragma unroll
                            for (int qi = 0; qi < 4; ++qi) {
                                two_sum_acc(s_re[warp][qi][0][s], s_re[warp][qi][1][s], r[qi][0]);
                                s_re[warp][qi][1][s] += r[qi][1];
                            }
                        }
                    }
#pragma unroll
                    for (int qi = 0; qi < 4; ++qi) {
                        two_sum_acc2(s_acc[qi][j][0][tid], s_acc[qi][j][1][tid], acc[qi][0]);
                        s_acc[qi][j][1][tid] = __fadd2_rn(s_acc[qi][j][1][tid], acc[qi][1]);
                    }
                }
                continue;
            }
            if (cls & kUnitSelf) {
                // a tile against its own chunks in the zero image: the one-sided units
#pragma unroll 1
                for (int j = 0; j < 2; ++j) {
                    const float* d0 = dl + 6 * (2 * j);
                    const float* d1 = dl + 6 * (2 * j + 1);
                    const float2 tx = s_th[0][j][tid], ty = s_th[1][j][tid], tz = s_th[2][j][tid];
                    if (!(cls & (j ? kUnitNear1 : kUnitNear0))) {
                        const float2 nx[1] = {make_float2(-(tx.x + d0[0]), -(tx.y + d1[0]))};
                        const float2 ny[1] = {make_float2(-(ty.x + d0[1]), -(ty.y + d1[1]))};
                        const float2 nz[1] = {make_float2(-(tz.x + d0[2]), -(tz.y + d1[2]))};
                        float2 aphi[1] = {make_float2(0.f, 0.f)}, agx[1] = {aphi[0]}, agy[1] = {aphi[0]},
                               agz[1] = {aphi[0]};
                        pair_loop_far<true, 1>(s_hi, nx, ny, nz, aphi, agx, agy, agz);
                        two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid], aphi[0]);
                        two_sum_acc2(s_acc[1][j][0][tid], s_acc[1][j][1][tid], agx[0]);
                        two_sum_acc2(s_acc[2][j][0][tid], s_acc[2][j][1][tid], agy[0]);
                        two_sum_acc2(s_acc[3][j][0][tid], s_acc[3][j][1][tid], agz[0]);
                        continue;
                    }
                    const int64_t i0 = (TA * kTgt32 + 2 * j) * kGroup + tid;
                    const int64_t i1 = i0 + kGroup;
                    const float4 C0 = a.pk_lo[2 * i0], D0 = a.pk_lo[2 * i0 + 1];
                    const float4 C1 = a.pk_lo[2 * i1], D1 = a.pk_lo[2 * i1 + 1];
                    const float2 tls[3] = {make_float2(C0.x, C1.x), make_float2(C0.z, C1.z), make_float2(D0.x, D1.x)};
                    const float2 ths[3] = {tx, ty, tz};
                    float2 nh[3], nl[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float e0, e1;
                        const float h0 = two_sum(ths[c].x, d0[c], e0);
                        const float h1 = two_sum(ths[c].y, d1[c], e1);
                        nh[c] = make_float2(-h0, -h1);
                        nl[c] = make_float2(-(e0 + (tls[c].x + d0[3 + c])), -(e1 + (tls[c].y + d1[3 + c])));
                    }
                    float2 aphi = make_float2(0.f, 0.f), aphi_lo = aphi, agx = aphi, agy = aphi, agz = aphi;
                    const float tau2 = S.tau2;
                    pair_loop_near<true>(s_hi, s_lo, nh[0], nh[1], nh[2], nl[0], nl[1], nl[2], aphi, aphi_lo, agx,
                                         agy, agz, tau2);
                    two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid], aphi);
                    s_acc[0][j][1][tid] = __fadd2_rn(s_acc[0][j][1][tid], aphi_lo);
                    two_sum_acc2(s_acc[1][j][0][tid], s_acc[1][j][1][tid], agx);
                    two_sum_acc2(s_acc[2][j][0][tid], s_acc[2][j][1][tid], agy);
                    two_sum_acc2(s_acc[3][j][0][tid], s_acc[3][j][1][tid], agz);
                }
                continue;
            }
            const float2 tq[2] = {s_tq[0][tid], s_tq[1][tid]};
            float2 agx[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, agy[2] = {agx[0], agx[0]},
                   agz[2] = {agx[0], agx[0]};
            float2 aphi[2] = {agx[0], agx[0]}, aphi2[2] = {agx[0], agx[0]};   // far: two interleaved sums; near: hi, lo
            if (kRefine && !(cls & kUnitNear)) {
                // refined potential terms (sym_far_step_pair_refined).  The targets' negated
                // offsets -(t + D) are rounded once from the float64 unit offset D = hi + lo; the
                // potential's running sums are cut every 8 steps: the action's two halves go into
                // the compensated sums, and each source's reaction is kept as four 8-step
                // segments (parked in registers while the sums rotate through the warp, then
                // fetched back by the lane that owns the source and added as a tree).
                float2 nx[4], ny[4], nz[4], c0[4], tq4[4], tqh4[4];
                float2 ph[4], pc[4], gx[4], gy[4], gz[4];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float* d0 = dl + 6 * (2 * j);
                    const float* d1 = dl + 6 * (2 * j + 1);
                    float o0[3], o1[3], w0 = 0.f, w1 = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        // n' = -(t + D) rounded once, and its remainder n'_lo
                        const float2 th = s_th[c][j][tid];
                        float e0, e1;
                        const float h0 = two_sum(th.x, d0[c], e0);
                        const float h1 = two_sum(th.y, d1[c], e1);
                        const float l0 = e0 + d0[3 + c], l1 = e1 + d1[3 + c];
                        float f0, f1;
                        o0[c] = -two_sum(h0, l0, f0);
                        o1[c] = -two_sum(h1, l1, f1);
                        w0 = fmaf(o0[c], -f0, w0);                    // n' . n'_lo
                        w1 = fmaf(o1[c], -f1, w1);
                    }
                    nx[2 * j] = make_float2(o0[0], o0[0]); nx[2 * j + 1] = make_float2(o1[0], o1[0]);
                    ny[2 * j] = make_float2(o0[1], o0[1]); ny[2 * j + 1] = make_float2(o1[1], o1[1]);
                    nz[2 * j] = make_float2(o0[2], o0[2]); nz[2 * j + 1] = make_float2(o1[2], o1[2]);
                    c0[2 * j] = make_float2(w0, w0); c0[2 * j + 1] = make_float2(w1, w1);
                    tq4[2 * j] = make_float2(tq[j].x, tq[j].x);
                    tq4[2 * j + 1] = make_float2(tq[j].y, tq[j].y);
                    tqh4[2 * j] = make_float2(-0.5f * tq[j].x, -0.5f * tq[j].x);      // exact
                    tqh4[2 * j + 1] = make_float2(-0.5f * tq[j].y, -0.5f * tq[j].y);
                }
#pragma unroll
                for (int i2 = 0; i2 < 4; ++i2) ph[i2] = pc[i2] = gx[i2] = gy[i2] = gz[i2] = make_float2(0.f, 0.f);
#pragma unroll 1
                for (int g = 0; g < nb64; ++g) {
                    float2 rp = make_float2(0.f, 0.f), rx = rp, ry = rp, rz = rp, st0 = rp, st1 = rp, st2 = rp;
#pragma unroll 1
                    for (int k = 0; k < 32; ++k) {
                        const int P = 32 * g + ((lane + k) & 31);
                        sym_far_step_pair_refined(s_sp[2 * P], s_sp[2 * P + 1], nx, ny, nz, c0, tq4, tqh4, ph, pc, gx,
                                                  gy, gz, rp, rx, ry, rz);
                        rp.x = __shfl_sync(0xffffffffu, rp.x, up);
                        rp.y = __shfl_sync(0xffffffffu, rp.y, up);
                        rx.x = __shfl_sync(0xffffffffu, rx.x, up);
                        rx.y = __shfl_sync(0xffffffffu, rx.y, up);
                        ry.x = __shfl_sync(0xffffffffu, ry.x, up);
                        ry.y = __shfl_sync(0xffffffffu, ry.y, up);
                        rz.x = __shfl_sync(0xffffffffu, rz.x, up);
                        rz.y = __shfl_sync(0xffffffffu, rz.y, up);
                        if ((k & 7) == 7) {
#pragma unroll
                            for (int j = 0; j < 2; ++j)
                                two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid],
                                             make_float2(ph[2 * j].x + ph[2 * j].y, ph[2 * j + 1].x + ph[2 * j + 1].y));
#pragma unroll
                            for (int i2 = 0; i2 < 4; ++i2) ph[i2] = make_float2(0.f, 0.f);
                            // after step k the lane holds pair (lane + k + 1) mod 32's partial sum
                            if (k == 7) st0 = rp;
                            if (k == 15) st1 = rp;
                            if (k == 23) st2 = rp;
                            if (k != 31) rp = make_float2(0.f, 0.f);
                        }
                    }
                    // pair lane's segments of steps 0-7, 8-15 and 16-23 sit 8, 16 and 24 lanes down
                    const float2 s1 = make_float2(__shfl_sync(0xffffffffu, st0.x, (lane + 24) & 31),
                                                  __shfl_sync(0xffffffffu, st0.y, (lane + 24) & 31));
                    const float2 s2 = make_float2(__shfl_sync(0xffffffffu, st1.x, (lane + 16) & 31),
                                                  __shfl_sync(0xffffffffu, st1.y, (lane + 16) & 31));
                    const float2 s3 = make_float2(__shfl_sync(0xffffffffu, st2.x, (lane + 8) & 31),
                                                  __shfl_sync(0xffffffffu, st2.y, (lane + 8) & 31));
                    const float2 tot = __fadd2_rn(__fadd2_rn(s1, s2), __fadd2_rn(s3, rp));
                    const int s = 64 * g + lane, sb = s + 32;    // the lane's pair: sources s, s + 32
                    two_sum_acc(s_re[warp][0][0][s], s_re[warp][0][1][s], tot.x);
                    two_sum_acc(s_re[warp][0][0][sb], s_re[warp][0][1][sb], tot.y);
                    two_sum_acc(s_re[warp][1][0][s], s_re[warp][1][1][s], rx.x);
                    two_sum_acc(s_re[warp][1][0][sb], s_re[warp][1][1][sb], rx.y);
                    two_sum_acc(s_re[warp][2][0][s], s_re[warp][2][1][s], ry.x);
                    two_sum_acc(s_re[warp][2][0][sb], s_re[warp][2][1][sb], ry.y);
                    two_sum_acc(s_re[warp][3][0][s], s_re[warp][3][1][s], rz.x);
                    two_sum_acc(s_re[warp][3][0][sb], s_re[warp][3][1][sb], rz.y);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    // the corrections (tiny against the terms, summed as -2x: scaled by -1/2, exact)
                    // into the low parts; the field as usual
                    s_acc[0][j][1][tid] = __fadd2_rn(s_acc[0][j][1][tid],
                                                     make_float2(-0.5f * (pc[2 * j].x + pc[2 * j].y),
                                                                 -0.5f * (pc[2 * j + 1].x + pc[2 * j + 1].y)));
                    two_sum_acc2(s_acc[1][j][0][tid], s_acc[1][j][1][tid],
                                 make_float2(gx[2 * j].x + gx[2 * j].y, gx[2 * j + 1].x + gx[2 * j + 1].y));
                    two_sum_acc2(s_acc[2][j][0][tid], s_acc[2][j][1][tid],
                                 make_float2(gy[2 * j].x + gy[2 * j].y, gy[2 * j + 1].x + gy[2 * j + 1].y));
                    two_sum_acc2(s_acc[3][j][0][tid], s_acc[3][j][1][tid],
                                 make_float2(gz[2 * j].x + gz[2 * j].y, gz[2 * j + 1].x + gz[2 * j + 1].y));
                }
                continue;
            }
            if (!(cls & kUnitNear)) {
                // targets as 4 scalars (duplicated into both halves), sources two at a time
                float2 nx[4], ny[4], nz[4], tq4[4];
                float2 ph[4], gx[4], gy[4], gz[4];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float* d0 = dl + 6 * (2 * j);
                    const float* d1 = dl + 6 * (2 * j + 1);
                    const float2 tx = s_th[0][j][tid], ty = s_th[1][j][tid], tz = s_th[2][j][tid];
                    const float a0 = -(tx.x + d0[0]), a1 = -(tx.y + d1[0]);
                    const float b0 = -(ty.x + d0[1]), b1 = -(ty.y + d1[1]);
                    const float c0 = -(tz.x + d0[2]), c1 = -(tz.y + d1[2]);
                    nx[2 * j] = make_float2(a0, a0); nx[2 * j + 1] = make_float2(a1, a1);
                    ny[2 * j] = make_float2(b0, b0); ny[2 * j + 1] = make_float2(b1, b1);
                    nz[2 * j] = make_float2(c0, c0); nz[2 * j + 1] = make_float2(c1, c1);
                    tq4[2 * j] = make_float2(tq[j].x, tq[j].x);
                    tq4[2 * j + 1] = make_float2(tq[j].y, tq[j].y);
                }
#pragma unroll
                for (int i2 = 0; i2 < 4; ++i2) ph[i2] = gx[i2] = gy[i2] = gz[i2] = make_float2(0.f, 0.f);
#pragma unroll 1
                for (int g = 0; g < nb64; ++g) {
                    float2 rp = make_float2(0.f, 0.f), rx = rp, ry = rp, rz = rp;
#pragma unroll 1
                    for (int k = 0; k < 32; ++k) {
                        const int P = 32 * g + ((lane + k) & 31);
                        sym_far_step_pair(s_sp[2 * P], s_sp[2 * P + 1], nx, ny, nz, tq4, ph, gx, gy, gz, rp, rx, ry,
                                          rz);
                        rp.x = __shfl_sync(0xffffffffu, rp.x, up);
                        rp.y = __shfl_sync(0xffffffffu, rp.y, up);
                        rx.x = __shfl_sync(0xffffffffu, rx.x, up);
                        rx.y = __shfl_sync(0xffffffffu, rx.y, up);
                        ry.x = __shfl_sync(0xffffffffu, ry.x, up);
                        ry.y = __shfl_sync(0xffffffffu, ry.y, up);
                        rz.x = __shfl_sync(0xffffffffu, rz.x, up);
                        rz.y = __shfl_sync(0xffffffffu, rz.y, up);
                    }
                    // the lane holds the reactions of pair 32 g + lane: sources s and s + 32
                    const int s = 64 * g + lane, s1 = s + 32;
                    two_sum_acc(s_re[warp][0][0][s], s_re[warp][0][1][s], rp.x);
                    two_sum_acc(s_re[warp][0][0][s1], s_re[warp][0][1][s1], rp.y);
                    two_sum_acc(s_re[warp][1][0][s], s_re[warp][1][1][s], rx.x);
                    two_sum_acc(s_re[warp][1][0][s1], s_re[warp][1][1][s1], rx.y);
                    two_sum_acc(s_re[warp][2][0][s], s_re[warp][2][1][s], ry.x);
                    two_sum_acc(s_re[warp][2][0][s1], s_re[warp][2][1][s1], ry.y);
                    two_sum_acc(s_re[warp][3][0][s], s_re[warp][3][1][s], rz.x);
                    two_sum_acc(s_re[warp][3][0][s1], s_re[warp][3][1][s1], rz.y);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    // the two sources' halves of each target's sums, folded once per unit
                    two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid],
                                 make_float2(ph[2 * j].x + ph[2 * j].y, ph[2 * j + 1].x + ph[2 * j + 1].y));
                    two_sum_acc2(s_acc[1][j][0][tid], s_acc[1][j][1][tid],
                                 make_float2(gx[2 * j].x + gx[2 * j].y, gx[2 * j + 1].x + gx[2 * j + 1].y));
                    two_sum_acc2(s_acc[2][j][0][tid], s_acc[2][j][1][tid],
                                 make_float2(gy[2 * j].x + gy[2 * j].y, gy[2 * j + 1].x + gy[2 * j + 1].y));
                    two_sum_acc2(s_acc[3][j][0][tid], s_acc[3][j][1][tid],
                                 make_float2(gz[2 * j].x + gz[2 * j].y, gz[2 * j + 1].x + gz[2 * j + 1].y));
                }
            } else {
                // near pairs present: every pair of the unit in float-float offsets
                float2 nh[2][3], nl[2][3];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float* d0 = dl + 6 * (2 * j);
                    const float* d1 = dl + 6 * (2 * j + 1);
                                        const int64_t i0 = (TA * kTgt32 + 2 * j) * kGroup + tid;
                    const int64_t i1 = i0 + kGroup;
                    const float4 C0 = a.pk_lo[2 * i0], D0 = a.pk_lo[2 * i0 + 1];
                    const float4 C1 = a.pk_lo[2 * i1], D1 = a.pk_lo[2 * i1 + 1];
                    const float2 tls[3] = {make_float2(C0.x, C1.x), make_float2(C0.z, C1.z), make_float2(D0.x, D1.x)};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 th = s_th[c][j][tid];
                        float e0, e1;
                        const float h0 = two_sum(th.x, d0[c], e0);
                        const float h1 = two_sum(th.y, d1[c], e1);
                        nh[j][c] = make_float2(-h0, -h1);
                        nl[j][c] = make_float2(-(e0 + (tls[c].x + d0[3 + c])), -(e1 + (tls[c].y + d1[3 + c])));
                    }
                }
#pragma unroll 1
                for (int g = 0; g < nb32; ++g) {
                    float rp = 0.f, rpl = 0.f, rx = 0.f, ry = 0.f, rz = 0.f;
#pragma unroll 1
                    for (int k0 = 0; k0 < 32; k0 += kNearFold) {
                        float2 blk[2];
#pragma unroll
                        for (int k = 0; k < kNearFold; ++k) {
                            sym_near_step(s_hi, s_lo, 32 * g + ((lane + k0 + k) & 31), nh, nl, tq, S.tau2, blk, k == 0,
                                          agx, agy, agz, rp, rpl, rx, ry, rz);
                            rp = __shfl_sync(0xffffffffu, rp, up);
                            rpl = __shfl_sync(0xffffffffu, rpl, up);
                            rx = __shfl_sync(0xffffffffu, rx, up);
                            ry = __shfl_sync(0xffffffffu, ry, up);
                            rz = __shfl_sync(0xffffffffu, rz, up);
                        }
#pragma unroll
                        for (int j = 0; j < 2; ++j) two_sum_acc2(aphi[j], aphi2[j], blk[j]);
                    }
                    const int s = 32 * g + lane;
                    two_sum_acc(s_re[warp][0][0][s], s_re[warp][0][1][s], rp);
                    s_re[warp][0][1][s] += rpl;
                    two_sum_acc(s_re[warp][1][0][s], s_re[warp][1][1][s], rx);
                    two_sum_acc(s_re[warp][2][0][s], s_re[warp][2][1][s], ry);
                    two_sum_acc(s_re[warp][3][0][s], s_re[warp][3][1][s], rz);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    two_sum_acc2(s_acc[0][j][0][tid], s_acc[0][j][1][tid], aphi[j]);
                    s_acc[0][j][1][tid] = __fadd2_rn(s_acc[0][j][1][tid], aphi2[j]);
                    two_sum_acc2(s_acc[1][j][0][tid], s_acc[1][j][1][tid], agx[j]);
                    two_sum_acc2(s_acc[2][j][0][tid], s_acc[2][j][1][tid], agy[j]);
                    two_sum_acc2(s_acc[3][j][0][tid], s_acc[3][j][1][tid], agz[j]);
                }
            }
        }
        if (!diag) {
            // the chunk's reaction: the warps' sums in a fixed order, into slot (tb, ta, gi) at
            // the chunk's positions in tile tb (the field with the reaction's sign)
            __syncthreads();
            const int64_t off = S.part0 + ((sym_slot(S, tb, ta) * S.n_g + gi) * 4) * kTile32;
            double* dst = a.partial + off + (chunk - c0) * kNearChunk;
            const bool ok = debug_in_range(off, 4 * kTile32, a.limit, a.status, a.n_status);
            for (int s = tid; s < kNearChunk && ok; s += kThreads32) {
#pragma unroll
                for (int qi = 0; qi < 4; ++qi) {
                    double v = 0.0;
#pragma unroll
                    for (int w = 0; w < kWarps; ++w) v += (double)s_re[w][qi][0][s] + (double)s_re[w][qi][1][s];
                    dst[qi * kTile32 + s] = qi == 0 ? v : -v;
                }
            }
        } else {
            // a tile against itself: the chunk is the tile's group k, and source s of it is this
            // thread's target in that group (pair k / 2, half k % 2); its reaction joins the
            // action sums, as hi + lo of the warps' sums in the same fixed order
            __syncthreads();
            const int k = (int)(chunk - c0), j = k >> 1;
#pragma unroll
            for (int qi = 0; qi < 4; ++qi) {
                double v = 0.0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) v += (double)s_re[w][qi][0][tid] + (double)s_re[w][qi][1][tid];
                if (qi) v = -v;
                const float vh = (float)v, vl = (float)(v - (double)vh);
                float2& h = s_acc[qi][j][0][tid];
                float2& l = s_acc[qi][j][1][tid];
                if (k & 1) {
                    two_sum_acc(h.y, l.y, vh);
                    l.y += vl;
                } else {
                    two_sum_acc(h.x, l.x, vh);
                    l.x += vl;
                }
            }
        }
    }
    // positions of tile tb past its last chunk (padding) get zero reactions, so that every
    // slot is defined
    if (!diag)
        for (int64_t c = c1; c < c0 + kTgt32; ++c) {
            const int64_t off = S.part0 + ((sym_slot(S, tb, ta) * S.n_g + gi) * 4) * kTile32;
            double* dst = a.partial + off + (c - c0) * kNearChunk;
            const bool ok = debug_in_range(off, 4 * kTile32, a.limit, a.status, a.n_status);
            for (int s = tid; s < kNearChunk && ok; s += kThreads32)
#pragma unroll
                for (int qi = 0; qi < 4; ++qi) dst[qi * kTile32 + s] = 0.0;
        }
    // the action on tile ta: slot (ta, tb, gi)
    {
        const int64_t off = S.part0 + ((sym_slot(S, ta, tb) * S.n_g + gi) * 4) * kTile32;
        double* dst = a.partial + off;
        const bool ok = debug_in_range(off, 4 * kTile32, a.limit, a.status, a.n_status);
#pragma unroll
        for (int qi = 0; qi < 4; ++qi)
#pragma unroll
            for (int j = 0; j < 2 && ok; ++j) {
                const float2 h = s_acc[qi][j][0][tid], l = s_acc[qi][j][1][tid];
                dst[qi * kTile32 + (2 * j) * kThreads32 + tid] = (double)h.x + (double)l.x;
                dst[qi * kTile32 + (2 * j + 1) * kThreads32 + tid] = (double)h.y + (double)l.y;
            }
    }
    }
}

// ---------------------------------------------------------------------------
// Symmetric float64 charge kernel: the float64 counterpart of k_near32s.  A tile of 128
// charges (one per thread) is also a source chunk; items are (tile pair (a <= b), image
// group); per image a warp visits the 128 sources of tile b in 4 rotations of 32, adding
// the action q_s / r to its targets and passing each source's reaction sums one lane down
// per step (float64 shuffles); every warp keeps its own float64 reaction sums per source,
// added in a fixed order when the item is done.  A tile against itself takes one image of
// each mirror pair with reactions onto its own charges, and the zero image one-sided.
// ---------------------------------------------------------------------------
struct Near64SymArgs {
    const double4_32a* pk;   // charges (x, y, z, q), absolute, padded with far-away zero charges
    const double* shifts;
    double* partial;         // per system [n_tiles][n_tiles * n_g][4][kTile64] from part0
    SymSysTable tab;
    int64_t W;
    int* counter;
    int* status;             // error words (debug bounds checks)
    int n_status;
    int64_t limit;           // doubles of the partial buffer (debug bounds checks)
};

template <int kMinB>
__global__ void __launch_bounds__(kThreads64, kMinB) k_near64s(Near64SymArgs a) {
    constexpr int kWarps = kThreads64 / 32;
    __shared__ double4_32a s_src[kNearChunk];
    __shared__ double s_re[kWarps][4][kNearChunk];   // reaction sums [warp][quantity][source]
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int up = (lane + 1) & 31;
    for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t item = s_item;
    __syncthreads();                     // every thread has the item (and is done with the last one)
    if (item >= a.W) break;
    const SymSys S = a.tab.many ? a.tab.many[sym_sys_by_item(a.tab, item)] : a.tab.one;
    const int64_t local = item - S.item0;
    const int64_t pair = local / S.n_g;
    const int gi = (int)(local - pair * S.n_g);
    int64_t ta, tb;
    sym_band_pair(S, pair, ta, tb);
    const bool diag = ta == tb;
    const int im0 = gi * S.img_per_g;
    const int nimg = min(S.img_per_g, S.n_img - im0);
    const double4_32a t = a.pk[(S.tile0 + ta) * kTile64 + tid];
    s_src[tid] = a.pk[(S.tile0 + tb) * kTile64 + tid];
#pragma unroll
    for (int qi = 0; qi < 4; ++qi)
#pragma unroll
        for (int k = 0; k < kNearChunk / 32; ++k) s_re[warp][qi][32 * k + lane] = 0.0;
    __syncthreads();
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    // the system's last tile holds last_n charges: source blocks of padding alone are skipped
    const int nb32 = tb == S.n_tiles - 1 && S.last_n > 0 ? (S.last_n + 31) >> 5 : kNearChunk / 32;
    for (int im = 0; im < nimg; ++im) {
        // y - x_i - p with the shift folded into the target
        const double* sh = a.shifts + 3 * (S.shift0 + im0 + im);
        const int sg = diag ? shift_sign(sh) : 1;
        if (sg < 0) continue;                    // a tile against itself: image -p by reaction
        const double px = t.x - sh[0], py = t.y - sh[1], pz = t.z - sh[2];
        if (sg == 0) {                           // ... and its zero image one-sided
#pragma unroll 4
            for (int s = 0; s < kNearChunk; ++s) {
                const double4_32a Q = s_src[s];
                const double ex = Q.x - px, ey = Q.y - py, ez = Q.z - pz;
                const double r2 = fma(ez, ez, fma(ey, ey, ex * ex));
                const double ri = rsqrt_f64_k0(r2);      // K(0) = 0
                const double qr = Q.w * ri;
                acc[0] += qr;
                const double w = qr * ri * ri;
                acc[1] = fma(ex, w, acc[1]);
                acc[2] = fma(ey, w, acc[2]);
                acc[3] = fma(ez, w, acc[3]);
            }
            continue;
        }
#pragma unroll 1
        for (int g = 0; g < nb32; ++g) {
            double rp = 0.0, rx = 0.0, ry = 0.0, rz = 0.0;
#pragma unroll 2
            for (int k = 0; k < 32; ++k) {
                const double4_32a Q = s_src[32 * g + ((lane + k) & 31)];
                const double ex = Q.x - px, ey = Q.y - py, ez = Q.z - pz;   // x_s + p - y
                const double r2 = fma(ez, ez, fma(ey, ey, ex * ex));
                const double ri = rsqrt_f64_k0(r2);
                const double ri2 = ri * ri;
                const double qa = Q.w * ri;              // action
                acc[0] += qa;
                const double wa = qa * ri2;
                acc[1] = fma(ex, wa, acc[1]);
                acc[2] = fma(ey, wa, acc[2]);
                acc[3] = fma(ez, wa, acc[3]);
                const double qb = t.w * ri;              // reaction (field sign folded later)
                rp += qb;
                const double wb = qb * ri2;
                rx = fma(ex, wb, rx);
                ry = fma(ey, wb, ry);
                rz = fma(ez, wb, rz);
                rp = __shfl_sync(0xffffffffu, rp, up);
                rx = __shfl_sync(0xffffffffu, rx, up);
                ry = __shfl_sync(0xffffffffu, ry, up);
                rz = __shfl_sync(0xffffffffu, rz, up);
            }
            const int s = 32 * g + lane;                 // the lane holds source s's reaction
            s_re[warp][0][s] += rp;
            s_re[warp][1][s] += rx;
            s_re[warp][2][s] += ry;
            s_re[warp][3][s] += rz;
        }
    }
    if (diag) {
        // a tile against itself: source tid is this thread's target, its reaction joins the action
        __syncthreads();
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) {
            double v = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) v += s_re[w][qi][tid];
            acc[qi] += qi == 0 ? v : -v;
        }
    }
    {
        const int64_t off = S.part0 + ((sym_slot(S, ta, tb) * S.n_g + gi) * 4) * kTile64;
        double* dst = a.partial + off + tid;
        if (debug_in_range(off, 4 * kTile64, a.limit, a.status, a.n_status))
#pragma unroll
            for (int qi = 0; qi < 4; ++qi) dst[qi * kTile64] = acc[qi];
    }
    if (!diag) {
        __syncthreads();
        const int64_t off = S.part0 + ((sym_slot(S, tb, ta) * S.n_g + gi) * 4) * kTile64;
        double* dst = a.partial + off + tid;
        const bool ok = debug_in_range(off, 4 * kTile64, a.limit, a.status, a.n_status);
#pragma unroll
        for (int qi = 0; qi < 4 && ok; ++qi) {
            double v = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) v += s_re[w][qi][tid];
            dst[qi * kTile64] = qi == 0 ? v : -v;
        }
    }
    }
}

// Reduction of the symmetric kernel's slots after one band: target i (packed order, i <
// n_valid) in tile t of its system adds the slots of row t that the band wrote -- for a band
// tile its block row and its actions on the tiles after the band, for a later tile its
// reactions from the band's tiles; tiles before the band have none -- each over the image
// groups.  A block takes 32 consecutive targets (one tile) and one quantity, its 8 warps every
// 8th slot, combined in a fixed order; `accumulate` adds to the output of the earlier bands.
template <int kTile>
__global__ void __launch_bounds__(32 * kReduceWarps) k_sym_reduce(const double* __restrict__ partial, int64_t n_valid,
                                                                 SymSysTable tab, double* __restrict__ out_phi,
                                                                 double* __restrict__ out_grad, int accumulate,
                                                                 int64_t limit, int* status, int n_status) {
    __shared__ double s_part[kReduceWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int qi = blockIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int64_t i = i0 + lane;
    const int64_t T = i0 / kTile;
    const SymSys S = tab.many ? tab.many[sym_sys_by_tile(tab, T)] : tab.one;
    const int64_t t = T - S.tile0;
    if (t < S.a0) return;                   // uniform over the block: no slot of this band
    const int64_t bw = S.a1 - S.a0, n_out = S.n_tiles - S.a1;
    // the row's slots as one or two contiguous runs of (slot, image group) entries
    int64_t r1, n1, r2 = 0, n2 = 0;
    if (t < S.a1) {
        r1 = sym_slot(S, t, S.a0);
        n1 = bw;
        r2 = n_out > 0 ? sym_slot(S, t, S.a1) : 0;
        n2 = n_out;
    } else {
        r1 = sym_slot(S, t, S.a0);
        n1 = bw;
    }
    const int64_t e1 = n1 * S.n_g, e_all = e1 + n2 * S.n_g;
    const int loc = (int)(i - T * kTile);
    const double* base = partial + S.part0 + qi * kTile + loc;
    double acc = 0.0;
    if (i < n_valid)
        for (int64_t k = warp; k < e_all; k += kReduceWarps) {
            const int64_t e = k < e1 ? r1 * S.n_g + k : r2 * S.n_g + (k - e1);
            if (debug_in_range(S.part0 + e * 4 * kTile, 4 * kTile, limit, status, n_status)) acc += base[e * 4 * kTile];
        }
    s_part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && i < n_valid) {
        double v = s_part[0][lane];
#pragma unroll
        for (int w = 1; w < kReduceWarps; ++w) v += s_part[w][lane];
        if (qi == 0) {
            out_phi[i] = accumulate ? out_phi[i] + v : v;
        } else if (out_grad) {
            double& o = out_grad[3 * i + qi - 1];
            o = accumulate ? o + v : v;
        }
    }
}

// size of the partial buffer as the debug bounds checks see it (a test may shrink it)
int64_t sym_limit(const NearSymLaunch& S) {
    const int64_t real = (int64_t)S.doubles;
    return S.debug_limit > 0 && S.debug_limit < real ? S.debug_limit : real;
}

constexpr int kNear32sMinBlocks = 4;
// the refined instance holds the offsets' low parts and the correction sums too
#ifndef PSUM_REFINED_MIN_BLOCKS
#define PSUM_REFINED_MIN_BLOCKS 4
#endif
constexpr int kNear32sRefMinBlocks = PSUM_REFINED_MIN_BLOCKS;

size_t near32s_dyn_smem(int img_per_g) {
    const size_t reaction = (size_t)(kThreads32 / 32) * 4 * 2 * kNearChunk * sizeof(float);
    return reaction + ((6 * kTgt32 * (size_t)img_per_g + img_per_g + 3) / 4) * sizeof(float4);
}

// the kernel's static and dynamic shared memory together pass the 48 KiB default: allow the
// largest dynamic size any image group needs
cudaError_t near32s_allow_smem() {
    const int bytes = (int)near32s_dyn_smem(kMaxImages);
    cudaError_t e = cudaFuncSetAttribute(k_near32s<kNear32sMinBlocks, false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_near32s<kNear32sRefMinBlocks, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_near32s<kNear32sMinBlocks, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
}

cudaError_t launch_near32s(const float4* pk_hi, const float4* pk_lo, const double* org, const float4* ext,
                           const double* shifts, double* partial, const NearSymLaunch& S, cudaStream_t st, bool ff,
                           bool refine) {
    if (!S.counter || !S.status || S.n_status < 1 || S.max_ipg < 1) return cudaErrorInvalidValue;
    if (S.W <= 0) return cudaSuccess;
    const cudaError_t ea = near32s_allow_smem();
    if (ea != cudaSuccess) return ea;
    Near32SymArgs a;
    a.pk_hi = pk_hi; a.pk_lo = pk_lo; a.org = org; a.ext = ext; a.shifts = shifts; a.partial = partial;
    a.tab = S.tab; a.W = S.W; a.max_ipg = S.max_ipg;
    a.counter = S.counter; a.status = S.status; a.n_status = S.n_status; a.inject = S.inject;
    a.limit = sym_limit(S);
    const cudaError_t e = cudaMemsetAsync(S.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const size_t smem = near32s_dyn_smem(S.max_ipg);
    if (ff)
        k_near32s<kNear32sMinBlocks, true, false><<<(unsigned)S.G, kThreads32, smem, st>>>(a);
    else if (refine)
        k_near32s<kNear32sRefMinBlocks, false, true><<<(unsigned)S.G, kThreads32, smem, st>>>(a);
    else
        k_near32s<kNear32sMinBlocks, false, false><<<(unsigned)S.G, kThreads32, smem, st>>>(a);
    return cudaGetLastError();
}

int near32s_occupancy_ctas(int img_per_g, bool ff, bool refine) {
    int nb = 0;
    near32s_allow_smem();
    const size_t smem = near32s_dyn_smem(img_per_g);
    if (ff)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_near32s<kNear32sMinBlocks, true, false>, kThreads32,
                                                      smem);
    else if (refine)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_near32s<kNear32sRefMinBlocks, false, true>, kThreads32,
                                                      smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_near32s<kNear32sMinBlocks, false, false>, kThreads32,
                                                      smem);
    return nb < 1 ? 1 : nb;
}

cudaError_t launch_sym_reduce(const double* partial, int64_t n_valid, const NearSymLaunch& S, double* out_phi,
                              double* out_grad, cudaStream_t st, bool fp64, bool accumulate) {
    if (n_valid <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((n_valid + 31) / 32), 4u);
    const int acc = accumulate ? 1 : 0;
    const int64_t lim = sym_limit(S);
    if (fp64)
        k_sym_reduce<kTile64><<<grid, 32 * kReduceWarps, 0, st>>>(partial, n_valid, S.tab, out_phi, out_grad, acc, lim,
                                                                S.status, S.n_status);
    else
        k_sym_reduce<kTile32><<<grid, 32 * kReduceWarps, 0, st>>>(partial, n_valid, S.tab, out_phi, out_grad, acc, lim,
                                                                S.status, S.n_status);
    return cudaGetLastError();
}

constexpr int kNear64sMinBlocks = 4;

cudaError_t launch_near64s(const double4_32a* pk, const double* shifts, double* partial, const NearSymLaunch& S,
                           cudaStream_t st) {
    if (!S.counter) return cudaErrorInvalidValue;
    if (S.W <= 0) return cudaSuccess;
    Near64SymArgs a;
    a.pk = pk; a.shifts = shifts; a.partial = partial; a.tab = S.tab; a.W = S.W; a.counter = S.counter;
    a.status = S.status; a.n_status = S.n_status; a.limit = sym_limit(S);
    const cudaError_t e = cudaMemsetAsync(S.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_near64s<kNear64sMinBlocks><<<(unsigned)S.G, kThreads64, 0, st>>>(a);
    return cudaGetLastError();
}

int near64s_occupancy_ctas() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_near64s<kNear64sMinBlocks>, kThreads64, 0);
    return nb < 1 ? 1 : nb;
}

}  // namespace psum
