// Device helpers and constants shared by the near-field kernels (near.cu: one-sided
// kernels; near_sym.cu: symmetric kernels): source-chunk staging by bulk copies on an
// mbarrier, compensated sums, the pair loops and the float-float primitives.
#pragma once

#include "launch.cuh"

namespace psum {


constexpr int kGroup = kNearChunk;             // points per origin group (= chunk size)
constexpr int kGroupsPerTile32 = kTile32 / kGroup;  // 4
static_assert(kThreads32 == kGroup, "one target per thread per group");
static_assert(kGroupsPerTile32 == kTgt32, "targets per thread = groups per tile");
static_assert(kTile64 == kNearChunk, "FP64 tile = one chunk");

// A unit is "near" when the distance between the target-group origin and the shifted
// chunk origin is at most kNearFactor times the sum of the two group radii.  Near units
// form the pair offsets from float-float (hi + lo) coordinates and honour K(0) = 0;
// far units cannot hold a pair closer than (kNearFactor - 1)(R_T + R_S), where the
// float32 offsets from the two origins are accurate to a few float32 ulps of the pair
// distance.  Measured at 1.5 / 1.25 / 1.0: charge kernel 110.2 / 108.3 / 107.7 ms at 1e5
// charges; potential error on four random workloads up to 4.1 / 4.7 / 5.7e-7, field error
// unchanged (1.7-2.1e-7).
constexpr double kNearFactor = 1.25;

__device__ __forceinline__ float rsqrt_mufu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Knuth's two-sum: s + err = a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float s = a + b;
    const float bp = s - a;
    err = (a - (s - bp)) + (b - bp);
    return s;
}



// ---------------------------------------------------------------------------
// Chunk staging by the bulk-copy (TMA) engine: one thread arms an mbarrier with the byte
// count and issues two cp.async.bulk copies (hi and lo parts, 4 KiB each) from global to
// shared memory; the CTA computes the chunk's image offsets meanwhile, and the same thread
// waits for the barrier's phase with an iteration limit.
// ---------------------------------------------------------------------------
constexpr int kChunkBytes = 2 * kNearChunk * (int)sizeof(float4);   // one of the two parts
constexpr long long kCopySpinLimit = 1LL << 22;   // polls; a copy lands in about a microsecond

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, int bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, int bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// true once the barrier has completed the phase with the given parity; false after the limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// unit classes against the ball S_b (flags in shared memory, per image of the staged chunk)
constexpr int kUnitNear0 = 1;      // the thread's target pair 0 (groups 0, 1): float-float offsets, K(0) = 0
constexpr int kUnitOutside = 2;    // every source image outside the ball: nothing to add
constexpr int kUnitStraddle = 4;   // per-source test against the ball
constexpr int kUnitNear1 = 8;      // the same for target pair 1 (groups 2, 3)
constexpr int kUnitNear = kUnitNear0 | kUnitNear1;
constexpr int kUnitWeighted = 16;  // while staging two-layer check sums: an image with a nonzero weight
// symmetric charge kernels, a tile against itself: the pairs of image -p come as the reactions
// of image p's, so of each mirror pair of nonzero images only the one whose first nonzero
// shift coordinate is positive runs (the other is skipped), and the zero image runs one-sided
constexpr int kUnitMirrored = 32;
constexpr int kUnitSelf = 64;

// +1, -1 or 0: the sign of the first nonzero coordinate of a shift (which of p and -p runs)
__device__ __forceinline__ int shift_sign(const double* sh) {
    return sh[0] != 0.0 ? (sh[0] > 0.0 ? 1 : -1)
                        : sh[1] != 0.0 ? (sh[1] > 0.0 ? 1 : -1) : sh[2] != 0.0 ? (sh[2] > 0.0 ? 1 : -1) : 0;
}

// |x + p|^2 <= Rb^2 with the rounding of a plain left-to-right evaluation (no contraction),
// the same decision for a source at the boundary as a straightforward float64 evaluation
__device__ __forceinline__ bool in_ball(double x0, double x1, double x2, const double* p, double Rb) {
    const double a = __dadd_rn(x0, p[0]), b = __dadd_rn(x1, p[1]), c = __dadd_rn(x2, p[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
    return r2 <= __dmul_rn(Rb, Rb);
}

#ifndef PSUM_FAR_UNROLL
#define PSUM_FAR_UNROLL 2
#endif
constexpr int kFarUnroll = PSUM_FAR_UNROLL;   // source pairs per unrolled step of the far loop

// Far units: one chunk of sources against the thread's 4 targets (2 packed pairs),
// plain float32 offsets s - t'.  One source: its potential terms into qr, its field
// terms added to the gradient sums.
template <bool kGrad, int NP>
__device__ __forceinline__ void pair_term(const float4* __restrict__ s_hi, int src, const float2 (&nx)[NP],
                                          const float2 (&ny)[NP], const float2 (&nz)[NP], float2 (&qr)[NP],
                                          float2 (&agx)[NP], float2 (&agy)[NP], float2 (&agz)[NP]) {
    const float4 A = s_hi[2 * src];       // x x y y
    const float4 B = s_hi[2 * src + 1];   // z z q q
    const float2 sq = make_float2(B.z, B.w);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float2 ex = __fadd2_rn(make_float2(A.x, A.y), nx[j]);
        const float2 ey = __fadd2_rn(make_float2(A.z, A.w), ny[j]);
        const float2 ez = __fadd2_rn(make_float2(B.x, B.y), nz[j]);
        float2 r2 = __fmul2_rn(ex, ex);
        r2 = __ffma2_rn(ey, ey, r2);
        r2 = __ffma2_rn(ez, ez, r2);
        const float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        qr[j] = __fmul2_rn(sq, ri);
        if (kGrad) {
            const float2 w = __fmul2_rn(qr[j], __fmul2_rn(ri, ri));
            agx[j] = __ffma2_rn(ex, w, agx[j]);
            agy[j] = __ffma2_rn(ey, w, agy[j]);
            agz[j] = __ffma2_rn(ez, w, agz[j]);
        }
    }
}

// NP packed target pairs (both of a thread's pairs, or one when its other pair is near)
template <bool kGrad, int NP>
__device__ __forceinline__ void pair_loop_far(const float4* __restrict__ s_hi, const float2 (&nx)[NP],
                                              const float2 (&ny)[NP], const float2 (&nz)[NP], float2 (&aphi)[NP],
                                              float2 (&agx)[NP], float2 (&agy)[NP], float2 (&agz)[NP],
                                              int n = kNearChunk) {
    // the potential, whose terms cancel most, goes into two partial sums, one over each half
    // of the sources: each runs over consecutive sources of the spatial order, whose signs
    // alternate in a lattice or in dipoles (even and odd sources apart would each sum one sign)
    float2 bphi[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) bphi[j] = make_float2(0.f, 0.f);
    const int hn = n >> 1;        // n is even (a chunk, or compacted sources in blocks of 4)
    if constexpr (!kGrad) {
        // potential only: each term q / r enters its sum by one fused multiply-add
#pragma unroll kFarUnroll
        for (int s = 0; s < hn; ++s) {
            const float4 A0 = s_hi[2 * s], B0 = s_hi[2 * s + 1];
            const float4 A1 = s_hi[2 * (s + hn)], B1 = s_hi[2 * (s + hn) + 1];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const float2 ex0 = __fadd2_rn(make_float2(A0.x, A0.y), nx[j]);
                const float2 ey0 = __fadd2_rn(make_float2(A0.z, A0.w), ny[j]);
                const float2 ez0 = __fadd2_rn(make_float2(B0.x, B0.y), nz[j]);
                const float2 ex1 = __fadd2_rn(make_float2(A1.x, A1.y), nx[j]);
                const float2 ey1 = __fadd2_rn(make_float2(A1.z, A1.w), ny[j]);
                const float2 ez1 = __fadd2_rn(make_float2(B1.x, B1.y), nz[j]);
                float2 r0 = __fmul2_rn(ex0, ex0), r1 = __fmul2_rn(ex1, ex1);
                r0 = __ffma2_rn(ey0, ey0, r0);
                r1 = __ffma2_rn(ey1, ey1, r1);
                r0 = __ffma2_rn(ez0, ez0, r0);
                r1 = __ffma2_rn(ez1, ez1, r1);
                aphi[j] = __ffma2_rn(make_float2(B0.z, B0.w), make_float2(rsqrt_mufu(r0.x), rsqrt_mufu(r0.y)), aphi[j]);
                bphi[j] = __ffma2_rn(make_float2(B1.z, B1.w), make_float2(rsqrt_mufu(r1.x), rsqrt_mufu(r1.y)), bphi[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) aphi[j] = __fadd2_rn(aphi[j], bphi[j]);
        return;
    }
#pragma unroll kFarUnroll
    for (int s = 0; s < hn; ++s) {
        float2 q0[NP], q1[NP];
        pair_term<kGrad, NP>(s_hi, s, nx, ny, nz, q0, agx, agy, agz);
        pair_term<kGrad, NP>(s_hi, s + hn, nx, ny, nz, q1, agx, agy, agz);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            aphi[j] = __fadd2_rn(aphi[j], q0[j]);
            bphi[j] = __fadd2_rn(bphi[j], q1[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) aphi[j] = __fadd2_rn(aphi[j], bphi[j]);
}

// (hi, lo) += v for a packed pair of accumulators: Knuth's two-sum with the error
// carried in lo.
__device__ __forceinline__ void two_sum_acc2(float2& hi, float2& lo, float2 v) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 s = __fadd2_rn(hi, v);
    const float2 bp = __ffma2_rn(m1, hi, s);              // s - hi
    const float2 t1 = __ffma2_rn(m1, bp, s);              // s - bp
    const float2 e1 = __ffma2_rn(m1, t1, hi);             // hi - (s - bp)
    const float2 e2 = __ffma2_rn(m1, bp, v);              // v - bp
    lo = __fadd2_rn(lo, __fadd2_rn(e1, e2));
    hi = s;
}

// Near units: one packed target pair at a time, offsets from hi + lo coordinates,
// K(0) = 0 applied.  They hold the closest pairs, whose large terms would dominate the
// rounding of a plain float32 running sum of the potential: blocks of kNearFold terms are
// summed in float32 and each block is added with its rounding error carried (two-sum into
// aphi, aphi_lo).
constexpr int kNearFold = 4;
static_assert(kNearChunk % kNearFold == 0, "whole blocks per chunk");

template <bool kGrad>
__device__ __forceinline__ void pair_loop_near(const float4* __restrict__ s_hi, const float4* __restrict__ s_lo,
                                               float2 nhx, float2 nhy, float2 nhz, float2 nlx, float2 nly,
                                               float2 nlz, float2& aphi, float2& aphi_lo, float2& agx, float2& agy,
                                               float2& agz, float tau2, int n = kNearChunk) {
#pragma unroll 1
    for (int s0 = 0; s0 < n; s0 += kNearFold) {
        float2 blk = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < kNearFold; ++k) {
            const int s = s0 + k;
            const float4 A = s_hi[2 * s];
            const float4 B = s_hi[2 * s + 1];
            const float4 C = s_lo[2 * s];
            const float4 D = s_lo[2 * s + 1];
            const float2 ex = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), nhx), __fadd2_rn(make_float2(C.x, C.y), nlx));
            const float2 ey = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), nhy), __fadd2_rn(make_float2(C.z, C.w), nly));
            const float2 ez = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), nhz), __fadd2_rn(make_float2(D.x, D.y), nlz));
            float2 r2 = __fmul2_rn(ex, ex);
            r2 = __ffma2_rn(ey, ey, r2);
            r2 = __ffma2_rn(ez, ez, r2);
            float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
            ri.x = r2.x > tau2 ? ri.x : 0.f;                  // K(0) = 0 (Eq. 1), coincident_r2 (psum_internal.cuh)
            ri.y = r2.y > tau2 ? ri.y : 0.f;
            const float2 qr = __fmul2_rn(make_float2(B.z, B.w), ri);
            blk = k == 0 ? qr : __fadd2_rn(blk, qr);
            if (kGrad) {
                const float2 w = __fmul2_rn(qr, __fmul2_rn(ri, ri));
                agx = __ffma2_rn(ex, w, agx);
                agy = __ffma2_rn(ey, w, agy);
                agz = __ffma2_rn(ez, w, agz);
            }
        }
        two_sum_acc2(aphi, aphi_lo, blk);
    }
}

// ---------------------------------------------------------------------------
// Float-float (FF) pair arithmetic: every quantity is an unevaluated sum hi + lo of two
// float32 values (about 44 significant bits), built from error-free transformations on
// the float32 pipe -- Knuth's two-sum and the fused-multiply-add product error -- so that
// float64-class results need no float64 pair arithmetic (a GB300 SM issues 1/64 as many
// float64 as float32 lane operations).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// s + e = a + b exactly
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2& e) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 s = __fadd2_rn(a, b);
    const float2 bp = __ffma2_rn(m1, a, s);              // s - a
    const float2 t1 = __ffma2_rn(m1, bp, s);             // s - bp
    const float2 e1 = __ffma2_rn(m1, t1, a);             // a - (s - bp)
    const float2 e2 = __ffma2_rn(m1, bp, b);             // b - bp
    e = __fadd2_rn(e1, e2);
    return s;
}

// (hi, lo) += (vh, vl)
__device__ __forceinline__ void ff_acc2(float2& hi, float2& lo, float2 vh, float2 vl) {
    float2 e;
    hi = two_sum2(hi, vh, e);
    lo = __fadd2_rn(lo, __fadd2_rn(vl, e));
}

// (ph, pl) = (ah, al) (bh, bl), dropping al bl
__device__ __forceinline__ float2 ff_mul2(float2 ah, float2 al, float2 bh, float2 bl, float2& pl) {
    const float2 ph = __fmul2_rn(ah, bh);
    float2 e = __ffma2_rn(ah, bh, neg2(ph));             // exact product error
    e = __ffma2_rn(ah, bl, e);
    pl = __ffma2_rn(al, bh, e);
    return ph;
}

// One chunk against one packed target pair t' (negated: nTh + nTl).  Source offsets
// s - t' come out of a two-sum of the hi parts plus the lo parts; r^2 is summed with
// the product errors; 1/r is the MUFU estimate y refined by one Newton step taken in
// float-float, ri = y - y (r^2 y^2 - 1)/2, which leaves a relative error near
// (3/2)(2^-22.9)^2 + 2^-46; K(0) = 0 where r^2 is zero or below tau2
// (coincident_r2 in psum_internal.cuh).  acc[q] = (hi, lo) of
// phi and (kGrad) the three field sums.
// The offset's hi part comes from the rounded target offset, so a pair closer than about one
// float32 ulp of the offsets (a few 1e-8 of the group size) has hi and lo parts of equal size
// and opposite sign, and r^2 formed from hi^2 + 2 hi lo is wrong; near units (kRenorm) first
// renormalise each component by a fast two-sum (3 more packed operations), far units cannot hold
// such a pair.
template <bool kRenorm>
__device__ __forceinline__ void ff_renorm(float2 (&eh)[3], float2 (&el)[3]) {
    if constexpr (kRenorm) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 sm = __fadd2_rn(eh[c], el[c]);
            el[c] = __fadd2_rn(el[c], neg2(__fadd2_rn(sm, neg2(eh[c]))));
            eh[c] = sm;
        }
    }
}

template <bool kGrad, bool kRenorm>
__device__ __forceinline__ void pair_loop_ff(const float4* __restrict__ s_hi, const float4* __restrict__ s_lo,
                                             const float2 (&nTh)[3], const float2 (&nTl)[3], float2 (&acc)[4][2],
                                             float tau2, int n = kNearChunk) {
#pragma unroll 1
    for (int s = 0; s < n; ++s) {
        const float4 A = s_hi[2 * s], B = s_hi[2 * s + 1], C = s_lo[2 * s], D = s_lo[2 * s + 1];
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
        // r^2 = sum (eh + el)^2 as r2h + r2l
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
        // 1/r
        const float2 y = make_float2(rsqrt_mufu(r2h.x), rsqrt_mufu(r2h.y));
        const float2 ah = __fmul2_rn(r2h, y);
        const float2 ae = __ffma2_rn(r2h, y, neg2(ah));       // r2h y = ah + ae
        const float2 bh = __fmul2_rn(ah, y);
        const float2 be = __ffma2_rn(ah, y, neg2(bh));        // ah y = bh + be
        float2 h = __fadd2_rn(bh, make_float2(-1.f, -1.f));   // exact: bh is within a factor 2 of 1
        h = __fadd2_rn(h, be);
        h = __ffma2_rn(ae, y, h);
        h = __ffma2_rn(__fmul2_rn(r2l, y), y, h);             // h = r^2 y^2 - 1
        float2 rih = y;
        float2 ril = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), y), h);
        if (!(r2h.x > tau2)) rih.x = ril.x = 0.f;             // K(0) = 0 (Eq. 1), coincident_r2 (psum_internal.cuh)
        if (!(r2h.y > tau2)) rih.y = ril.y = 0.f;
        // q / r
        float2 Pl;
        const float2 Ph = ff_mul2(qh, ql, rih, ril, Pl);
        ff_acc2(acc[0][0], acc[0][1], Ph, Pl);
        if (kGrad) {
            // w = q / r^3, field term w (s - t')
            float2 r2il;
            const float2 r2ih = ff_mul2(rih, ril, rih, ril, r2il);
            float2 wl;
            const float2 wh = ff_mul2(Ph, Pl, r2ih, r2il, wl);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 gl;
                const float2 gh = ff_mul2(wh, wl, eh[c], el[c], gl);
                ff_acc2(acc[1 + c][0], acc[1 + c][1], gh, gl);
            }
        }
    }
}

// 1/sqrt(r2), or 0 for r2 = 0 (K(0) = 0, Eq. 1), in float64.  MUFU estimate y0 (relative
// error below 2^-22), then one third-order correction: with e = 1 - r2 y0^2,
// 1/sqrt(r2) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + O(e^3)), whose truncation
// (5/16)|e|^3 < 1e-20 is below float64 rounding; 5 float64 operations where two
// Newton-Raphson steps take 7.  The conversions between float64 and float32 around the
// MUFU estimate are done on the bit patterns with integer operations (the float64 pipe, which
// bounds this kernel, also runs the conversion instructions): the float32 copy of r2 keeps
// the top 23 mantissa bits (truncated, relative error below 2^-23, so |e| < 2^-21 and the
// correction's truncation stays below 1e-19), the estimate is widened exactly.  The zero test
// is taken on that float32 copy (a float32 compare and selects instead of a float64 compare);
// r2 below 2^-126 counts as zero, which would need two distinct charges within 1e-19 of each
// other.
__device__ __forceinline__ double rsqrt_f64_k0(double r2) {
    // float32 bits: the float64 exponent rebiased (1023 -> 127) and the mantissa cut to 23 bits
    const long long t = (__double_as_longlong(r2) >> 29) - (896LL << 23);
    const float r2f = __int_as_float(t > 0 ? (int)t : 0);
    const float yf = rsqrt_mufu(r2f);
    // float64 bits of the (positive, normal) estimate: exponent rebiased, mantissa widened
    const double y = __longlong_as_double(((long long)__float_as_int(yf) << 29) + (896LL << 52));
    const double e = fma(-r2, y * y, 1.0);
    const double ri = fma(y * e, fma(0.375, e, 0.5), y);
    return r2f > 0.f ? ri : 0.0;
}

// Debug builds (-DPSUM_DEBUG_CHECKS=1) check every write and read of the pair kernels'
// partial sums against the buffer's size: an access outside it is skipped and flagged in the
// launch's status words (kStatBounds, PSUM_ERR_INTERNAL at psum_sync) instead of faulting.
__device__ __forceinline__ bool debug_in_range(int64_t off, int64_t n, int64_t limit, int* status, int n_status) {
#if PSUM_DEBUG_CHECKS
    if (off < 0 || off + n > limit) {
        for (int k = 0; k < n_status; ++k) atomicOr(status + k, kStatBounds);
        return false;
    }
#endif
    return true;
}

// warps of the reduction kernels (fixed-order combination of the partial slots)
constexpr int kReduceWarps = 8;

}  // namespace psum
