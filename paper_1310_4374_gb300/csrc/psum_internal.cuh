// Internal definitions shared by the psum translation units (product code).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "psum.h"

namespace psum {

// ---------------------------------------------------------------------------
// Tiling of the near-field pair sum.
//   * a source CHUNK is kNearChunk consecutive (Hilbert-ordered) sources staged
//     in shared memory, with one float64 origin;
//   * a target TILE is kThreads threads x kTgt targets, with one float64 origin;
//   * a work UNIT is (tile, chunk, image): every target of the tile against
//     every source of the chunk shifted by one image vector.
// ---------------------------------------------------------------------------
constexpr int kNearChunk = 128;           // sources per chunk (both precisions)
constexpr int kThreads32 = 128;           // threads per CTA, FP32C kernel
constexpr int kTgt32 = 4;                 // targets per thread, FP32C kernel (2 packed pairs)
constexpr int kTile32 = kThreads32 * kTgt32;
constexpr int kThreads64 = 128;           // threads per CTA, FP64 kernel
constexpr int kTile64 = kThreads64;       // one target per thread
constexpr int kMaxImages = 343;           // K <= 3 per axis; trimmed plans: images kept
constexpr int kMaxDegree = 40;

// Spatial order of the charges: the index of a point's cell of a 256^3 grid over the box along
// the 3-D Hilbert curve (24 bits), computed by Skilling's method ("Programming the Hilbert
// curve", AIP Conf. Proc. 707, 2004): the cell's coordinates are turned in place into the
// curve's "transposed" index (undoing the excess rotations level by level, then a Gray code),
// whose bits interleaved level by level, axis 0 first, give the index.  Consecutive cells of
// the curve share a face, so groups of consecutive points are compact (a Z-order curve jumps
// between distant cells; its groups' bounding boxes are larger and more pairs of groups are
// near one another).
__host__ __device__ __forceinline__ uint32_t spread3_8(uint32_t v) {
    // 8 bits -> every third bit of 24
    v &= 0xffu;
    v = (v | (v << 8)) & 0x00f00fu;
    v = (v | (v << 4)) & 0x0c30c3u;
    v = (v | (v << 2)) & 0x249249u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t hilbert_key24(uint32_t c0, uint32_t c1, uint32_t c2) {
    uint32_t X[3] = {c0 & 0xffu, c1 & 0xffu, c2 & 0xffu};
    for (uint32_t Q = 1u << 7; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;                                 // invert the low bits of axis 0
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;      // exchange the low bits of axes 0 and i
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = 1u << 7; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    return (spread3_8(X[0]) << 2) | (spread3_8(X[1]) << 1) | spread3_8(X[2]);
}

// two-layer check points: flag in a group's class mask for a group of padding alone
constexpr int kGroupEmpty = 1 << 30;

// device status bits (OR-ed by kernels, mapped to PSUM_ERR_* on the host)
constexpr int kStatNonNeutral = 1;
constexpr int kStatOutOfBox = 2;
constexpr int kStatNonFinite = 4;
constexpr int kStatTimeout = 8;
constexpr int kStatBounds = 16;    // a debug-build bounds check refused an access (PSUM_DEBUG_CHECKS)
#ifndef PSUM_DEBUG_CHECKS
#define PSUM_DEBUG_CHECKS 0        // 1: range checks on the pair kernels' partial sums
#endif

// 0-based stacking of Eq. 1.8: t = n(n+1) + m
__host__ __device__ __forceinline__ int sh_index(int n, int m) { return n * (n + 1) + m; }

// ---------------------------------------------------------------------------
// Renormalised regular solid harmonics R^_n^m(u) (Eqs. 1.6-1.7), written as a
// recurrence directly on R^ so that the factorials never appear:
//   R^_0^0 = 1
//   R^_m^m   = -(x a + y b) sqrt((2m-1)/(2m)),  R^_m^-m = (y a - x b) sqrt((2m-1)/(2m)),
//              a = R^_{m-1}^{m-1}, b = R^_{m-1}^{-(m-1)}  (b = 0 for m = 1)
//   R^_{m+1}^{+-m} = -z sqrt(2m+1) R^_m^{+-m}
//   R^_n^{+-m} = -[(2n-1) z R^_{n-1} / sqrt((n-m)(n+m))
//                  + r^2 sqrt((n-m-1)(n+m-1)/((n-m)(n+m))) R^_{n-2}]
// (Eq. 1.6 with each factor sqrt((n-m)!(n+m)!) of Eq. 1.7 divided out step by step).
// The visitor is called once per (n, m) with the value and its gradient.
// ---------------------------------------------------------------------------
template <bool kGrad, class Visit>
__host__ __device__ __forceinline__ void sh_visit(double x, double y, double z, int p, Visit&& visit) {
    const double r2 = x * x + y * y + z * z;
    // sectoral pair (m, -m) carried along the diagonal, with gradients
    double a = 1.0, b = 0.0;
    double ax = 0, ay = 0, az = 0, bx = 0, by = 0, bz = 0;
    for (int m = 0; m <= p; ++m) {
        double sp, sm, spx = 0, spy = 0, spz = 0, smx = 0, smy = 0, smz = 0;
        if (m == 0) {
            sp = 1.0;
            sm = 0.0;
        } else {
            const double c = sqrt((2.0 * m - 1.0) / (2.0 * m));
            sp = -(x * a + y * b) * c;
            sm = (y * a - x * b) * c;
            if (kGrad) {
                spx = -(a + x * ax + y * bx) * c;
                spy = -(x * ay + b + y * by) * c;
                spz = -(x * az + y * bz) * c;
                smx = (y * ax - b - x * bx) * c;
                smy = (a + y * ay - x * by) * c;
                smz = (y * az - x * bz) * c;
            }
        }
        a = sp; b = sm;
        if (kGrad) { ax = spx; ay = spy; az = spz; bx = smx; by = smy; bz = smz; }
        // walk up in n for +m and -m
        for (int s = 0; s < (m == 0 ? 1 : 2); ++s) {
            const int mm = s == 0 ? m : -m;
            double v2 = s == 0 ? sp : sm;            // R^_m^mm
            double g2x = s == 0 ? spx : smx, g2y = s == 0 ? spy : smy, g2z = s == 0 ? spz : smz;
            visit(m, mm, v2, g2x, g2y, g2z);
            if (m + 1 > p) continue;
            const double c1 = sqrt(2.0 * m + 1.0);
            double v1 = -z * c1 * v2;                 // R^_{m+1}^mm
            double g1x = 0, g1y = 0, g1z = 0;
            if (kGrad) {
                g1x = -z * c1 * g2x;
                g1y = -z * c1 * g2y;
                g1z = -c1 * (v2 + z * g2z);
            }
            visit(m + 1, mm, v1, g1x, g1y, g1z);
            for (int n = m + 2; n <= p; ++n) {
                const double nm = (double)(n - m) * (double)(n + m);
                const double e1 = (2.0 * n - 1.0) / sqrt(nm);
                const double e2 = sqrt((double)(n - m - 1) * (double)(n + m - 1) / nm);
                const double v = -(e1 * z * v1 + e2 * r2 * v2);
                double gx = 0, gy = 0, gz = 0;
                if (kGrad) {
                    gx = -(e1 * z * g1x + e2 * (2.0 * x * v2 + r2 * g2x));
                    gy = -(e1 * z * g1y + e2 * (2.0 * y * v2 + r2 * g2y));
                    gz = -(e1 * (v1 + z * g1z) + e2 * (2.0 * z * v2 + r2 * g2z));
                }
                visit(n, mm, v, gx, gy, gz);
                v2 = v1; v1 = v;
                if (kGrad) { g2x = g1x; g2y = g1y; g2z = g1z; g1x = gx; g1y = gy; g1z = gz; }
            }
        }
    }
}

// The same recurrence with its coefficients read from a table, in value type T
// (double, or float for the FP32C far field).  Table layout for degree p:
//   [0, p]           c_m  = sqrt((2m-1)/(2m))   (m >= 1; c_0 unused)
//   [p+1, 2p+1]      c1_m = sqrt(2m+1)
//   then e1(n,m) = (2n-1)/sqrt((n-m)(n+m)) and e2(n,m) = sqrt((n-m-1)(n+m-1)/((n-m)(n+m)))
//   for 0 <= m <= n <= p at 2p+2 + 2 (n(n+1)/2 + m) and the entry after it.
__host__ __device__ __forceinline__ int sh_tab_size(int p) { return 2 * (p + 1) + (p + 1) * (p + 2); }

inline void sh_tab_fill(int p, double* t) {
    for (int m = 0; m <= p; ++m) {
        t[m] = m == 0 ? 0.0 : std::sqrt((2.0 * m - 1.0) / (2.0 * m));
        t[p + 1 + m] = std::sqrt(2.0 * m + 1.0);
    }
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            double* e = t + 2 * (p + 1) + 2 * (n * (n + 1) / 2 + m);
            const double nm = (double)(n - m) * (double)(n + m);
            e[0] = nm > 0 ? (2.0 * n - 1.0) / std::sqrt(nm) : 0.0;
            e[1] = nm > 0 ? std::sqrt((double)(n - m - 1) * (double)(n + m - 1) / nm) : 0.0;
        }
}

template <bool kGrad, class T, class Visit>
__host__ __device__ __forceinline__ void sh_visit_tab(T x, T y, T z, int p, const T* __restrict__ tab,
                                                      Visit&& visit) {
    const T r2 = x * x + y * y + z * z;
    const T* e12 = tab + 2 * (p + 1);
    T a = T(1), b = T(0);
    T ax = 0, ay = 0, az = 0, bx = 0, by = 0, bz = 0;
    for (int m = 0; m <= p; ++m) {
        T sp, sm, spx = 0, spy = 0, spz = 0, smx = 0, smy = 0, smz = 0;
        if (m == 0) {
            sp = T(1);
            sm = T(0);
        } else {
            const T c = tab[m];
            sp = -(x * a + y * b) * c;
            sm = (y * a - x * b) * c;
            if (kGrad) {
                spx = -(a + x * ax + y * bx) * c;
                spy = -(x * ay + b + y * by) * c;
                spz = -(x * az + y * bz) * c;
                smx = (y * ax - b - x * bx) * c;
                smy = (a + y * ay - x * by) * c;
                smz = (y * az - x * bz) * c;
            }
        }
        a = sp; b = sm;
        if (kGrad) { ax = spx; ay = spy; az = spz; bx = smx; by = smy; bz = smz; }
        for (int s = 0; s < (m == 0 ? 1 : 2); ++s) {
            const int mm = s == 0 ? m : -m;
            T v2 = s == 0 ? sp : sm;
            T g2x = s == 0 ? spx : smx, g2y = s == 0 ? spy : smy, g2z = s == 0 ? spz : smz;
            visit(m, mm, v2, g2x, g2y, g2z);
            if (m + 1 > p) continue;
            const T c1 = tab[p + 1 + m];
            T v1 = -z * c1 * v2;
            T g1x = 0, g1y = 0, g1z = 0;
            if (kGrad) {
                g1x = -z * c1 * g2x;
                g1y = -z * c1 * g2y;
                g1z = -c1 * (v2 + z * g2z);
            }
            visit(m + 1, mm, v1, g1x, g1y, g1z);
            for (int n = m + 2; n <= p; ++n) {
                const T* e = e12 + 2 * (n * (n + 1) / 2 + m);
                const T e1 = e[0], e2 = e[1];
                const T v = -(e1 * z * v1 + e2 * r2 * v2);
                T gx = 0, gy = 0, gz = 0;
                if (kGrad) {
                    gx = -(e1 * z * g1x + e2 * (T(2) * x * v2 + r2 * g2x));
                    gy = -(e1 * z * g1y + e2 * (T(2) * y * v2 + r2 * g2y));
                    gz = -(e1 * (v1 + z * g1z) + e2 * (T(2) * z * v2 + r2 * g2z));
                }
                visit(n, mm, v, gx, gy, gz);
                v2 = v1; v1 = v;
                if (kGrad) { g2x = g1x; g2y = g1y; g2z = g1z; g1x = gx; g1y = gy; g1z = gz; }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The plan (algorithm "set" results, device copies and scratch).
// ---------------------------------------------------------------------------
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct Plan {
    psum_opts opt{};
    int device = 0;
    int P = 0;                  // (p+1)^2
    double R0 = 0;
    double lambda_eff = 0;
    double Rb = 0;                  // > 0: near set trimmed to the ball of this radius
    double cond_est = 0;
    int rank = 0;
    int n_images = 0;
    std::vector<double> shifts;     // n_images x 3: image vectors (i1 d1, i2 d2, i3 d3)
    std::vector<double> Y, Yt;      // M x 3 check points and partners
    std::vector<double> pinv;       // (P-1) x M pseudo-inverse of A (row-major)
    std::vector<double> Rbox;       // P box integrals R_t^(0)
    std::vector<double> Xs;         // RBF basis: n_rbf centres x 3
    // a stored factorisation (psum_plan_load): when preset_pinv is not empty, algorithm "set"
    // takes it instead of factoring A, after checking that the geometry hashes the same
    std::vector<double> preset_pinv;
    int preset_rank = 0;
    double preset_cond = 0.0;
    uint64_t preset_geom = 0;
    uint64_t geom_hash = 0;         // FNV-1a of the check points and their partners (bit patterns)
    int self_image = 0;             // index of the zero image vector in `shifts`

    // check targets (2M points) as the near kernels consume them
    int n_check = 0;                // 2M
    int n_check_tiles = 0;
    int check_tile = 0;             // targets per check tile
    int* d_check_pos = nullptr;     // 2M: position of target j (j < M: y_j, else y~_{j-M}) in the packed order
    int* d_check_inv = nullptr;     // packed position -> j (-1 for padding), FP32C only
    void* d_check_tgt = nullptr;    // packed check targets (float4 rel coords or double4_32a)
    double* d_check_org = nullptr;  // tile origins (FP32C), 3 per tile

    // the right-hand side as two image layers at the M check points (PSUM_CHECKS_LAYERS):
    // f_l = sum over the layer i_k = s(K_k + 1) minus the layer i_k = -s K_k, where the
    // partner is y~_l = y_l - s d_k e_k.  Points of one class c = 2k + (s < 0) share their
    // image list; each packed point carries its class in the (unused) charge slot.
    int lc_tiles = 0;               // target tiles (0: the plan evaluates the 2M points)
    int lc_img = 0;                 // images per class: 2 x the largest layer (zero-weight padding)
    void* d_lc_tgt = nullptr;       // packed points (class in the charge slot): float32 hi parts then lo parts, or double4_32a
    double* d_lc_org = nullptr;     // float32 packing: 4 per group, origin and radius
    int* d_lc_gmask = nullptr;      // float32 packing: the classes present in each group (bit mask)
    double* d_lc_sub = nullptr;     // float32 packing: [group][6][4] centre and radius of each class's points
    int* d_lc_pos = nullptr;        // M: packed position of y_l
    double* d_lc_shifts = nullptr;  // [6][lc_img][3] image vectors of each class's layers
    float* d_lc_w = nullptr;        // [6][lc_img] weights: +1 (upper layer), -1 (lower), 0 (padding)

    // the backward's check sources as two image layers (float32 packing, plans with layers):
    // psi(x) = sum_l u_l [G(y~_l - x) - G(y_l - x)] is, as f_l, the sum over the two layers of
    // class c(l) with signs +-1, so each check point is a source of charge +u_l with the upper
    // layer's images and one of -u_l with the lower layer's (negated: the point is the source).
    // The 12 (class, side) sets are packed set by set in whole chunks of 128; each chunk has its
    // image list (bk_img0: first entry of d_bk_shifts) and count (bk_nimg).
    int bk_chunks = 0;              // 0: the backward keeps the 2M check points as sources
    int bk_lmax = 0;                // images per (class, side) list
    void* d_bk_pk = nullptr;        // float4 hi parts (2 per slot) then lo parts; charges set per backward
    double* d_bk_org = nullptr;     // 4 per chunk: origin and radius
    int* d_bk_slot = nullptr;       // per slot: 2 l + (lower side), or -1 for padding
    int* d_bk_img0 = nullptr;       // per chunk
    int* d_bk_nimg = nullptr;       // per chunk
    double* d_bk_shifts = nullptr;  // [12][bk_lmax][3]

    double* d_pinv = nullptr;
    double* d_Rbox = nullptr;
    double* d_shtab64 = nullptr;    // recurrence coefficients (sh_visit_tab), double
    float* d_shtab32 = nullptr;     // the same in float
    double* d_shifts = nullptr;
    double* d_rbf = nullptr;        // RBF basis: the n_rbf centres, 3 each
    double* d_C = nullptr;          // P coefficients of the last evaluation
    int* d_status = nullptr;
    int* h_status = nullptr;        // pinned

    // test hook: bytes of symmetric-kernel partial slots per band (0: kSymBandBytes)
    size_t sym_band_bytes = 0;

    // scratch, grown on demand
    DevBuf scratch;
    // pinned host staging and device staging for psum_eval_host
    DevBuf dstage;

    int num_sms = 0;
};

// ---------------------------------------------------------------------------
// Host helpers implemented in plan.cu
// ---------------------------------------------------------------------------
int build_plan(const psum_opts& o, Plan& pl);     // algorithm "set" on the host, then upload
void free_plan_device(Plan& pl);

// ---------------------------------------------------------------------------
// Equal contiguous ranges of the (tile, chunk, image) unit space: range g of G covers units
// [bound(g), bound(g+1)), bound(g) = floor(g U / G).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t sk_bound(int64_t g, int64_t U, int64_t G) {
    return (g * U) / G;
}
// the CTA whose range contains unit u
__host__ __device__ __forceinline__ int64_t sk_owner(int64_t u, int64_t U, int64_t G) {
    // largest g with floor(g U / G) <= u  <=>  g U < (u + 1) G
    int64_t g = ((u + 1) * G - 1) / U;
    if (g > G - 1) g = G - 1;
    return g;
}

// One system of a near-field launch.  Its work units are the global indices
// [unit0, unit0 + n_tiles * n_chunks * n_img), ordered (tile, chunk, image).
// Two charges at one position but in different groups: their float32 and float-float offsets
// come from two different group origins and carry a few 2^-48 of the group scale in rounding,
// so the pair comes out a tiny, nonzero distance apart and its 1/r is meaningless.  The near
// units (and every float-float unit) take a pair closer than 2^-37 R0 (R0 the half diagonal of
// the box, which bounds the group radii) as coincident, K(0) = 0 as for an exact zero (Eq. 1);
// float32 offsets resolve no distance that small anyway.  The squared threshold, per system.
inline float coincident_r2(const double d[3]) {
    const double t = std::ldexp(0.5 * std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), -37);
    return (float)(t * t);
}

struct NearSys {
    int64_t unit0;       // first unit
    int64_t tile0;       // first tile of the system in the target pack (= its first partial-buffer row)
    int64_t n_tiles;     // target tiles
    int64_t n_chunks;    // source chunks
    int64_t src_chunk0;  // first chunk of the system in the source pack
    int shift0;          // first image vector of the system in the shift table
    int n_img;
    int64_t chunk_stride;  // a tile visits its chunks in the order (k * chunk_stride) mod n_chunks
    float tau2;          // coincident_r2 of the system's box (float32 kernels)
};

// A stride near n / golden ratio, coprime to n: consecutive steps land far apart in the
// (Hilbert-ordered) chunk sequence, so the chunks next to a tile -- the costly float-float
// "near" units -- spread evenly over the work items instead of
// piling up in the few whose unit ranges hold the tile's spatial neighbours.
inline int64_t near_chunk_stride(int64_t n) {
    if (n <= 2) return 1;
    int64_t s = (int64_t)(0.6180339887498949 * (double)n);
    if (s < 1) s = 1;
    auto gcd = [](int64_t a, int64_t b) {
        while (b) {
            const int64_t t = a % b;
            a = b;
            b = t;
        }
        return a;
    };
    while (gcd(s, n) != 1) ++s;
    return s;
}

// A single system travels by value; a batch passes a device array sorted by unit0.
struct NearSysTable {
    NearSys one;
    const NearSys* many;   // nullptr: the launch has the single system `one`
    int n;
};

__host__ __device__ __forceinline__ int64_t near_sys_units(const NearSys& s) {
    return s.n_tiles * s.n_chunks * s.n_img;
}

__device__ __forceinline__ NearSys near_sys_get(const NearSysTable& t, int b) {
    return t.many ? t.many[b] : t.one;
}

// the system whose unit range contains u (binary search over unit0)
__device__ __forceinline__ int near_sys_by_unit(const NearSysTable& t, int64_t u) {
    if (!t.many) return 0;
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.many[mid].unit0 <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// the system whose partial-buffer rows contain global tile T
__device__ __forceinline__ int near_sys_by_tile(const NearSysTable& t, int64_t T) {
    if (!t.many) return 0;
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.many[mid].tile0 <= T) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The unit space is cut into W equal contiguous work items (fixed ranges, so every tile's
// partial slots and every summation order are fixed: results are bitwise reproducible);
// G resident CTAs take items in order from a device counter.  Co-resident CTAs of an SM
// progress at different rates (measured: 47-130 ms for equal shares of one 130 ms
// launch), so a static share per CTA left SMs under-occupied for half the launch.  16
// items per CTA: the tail is at most one small item; the partial sums grow with the
// item count (16 KiB per item and tile) and their reduction stays under 1 ms at 1e5 charges.
#ifndef PSUM_ITEMS_PER_CTA
#define PSUM_ITEMS_PER_CTA 16
#endif
constexpr int kItemsPerCta = PSUM_ITEMS_PER_CTA;
// The check-point launch has few target tiles (M or 2M points): 2 items per CTA keep its
// partial sums (and their reduction) small; 1, 2, 4 and 16 measured within 0.3% end to end.
#ifndef PSUM_CHECK_ITEMS_PER_CTA
#define PSUM_CHECK_ITEMS_PER_CTA 2
#endif
constexpr int kCheckItemsPerCta = PSUM_CHECK_ITEMS_PER_CTA;
constexpr int64_t kMinUnitsPerItem = 32;

struct NearPlanLaunch {
    int64_t U, G;
    int64_t W;                    // work items
    int* counter = nullptr;       // device int, zeroed by the launcher before each launch
    int* status = nullptr;        // device error words the pair kernel may flag (kStatTimeout)
    int n_status = 0;
    int inject = 0;               // test hook: arm the chunk-copy barrier for bytes that never come
    int64_t debug_limit = 0;      // test hook of the debug bounds checks: a smaller partial buffer (doubles)
    int max_contrib;              // partial slots per tile
    int max_img;                  // largest image count of any system (shared-memory sizing)
    int64_t n_tiles;              // rows of the partial buffer
    NearSysTable tab;
};

// The symmetric charge kernel (FP32C, block image sets): work items are (system, tile pair
// (a <= b), group of images).  The targets are the system's charges, packed in whole tiles from
// global tile tile0 (groups 4 tile0 ..); its source chunks are the first n_chunks groups.
//
// Partial sums: the action of pair (a, b) on tile a and its reaction on tile b each go to a slot
// of 4 x tile doubles per image group, one writer per slot.  A launch covers the BAND of row
// tiles a0 <= a < a1 (pairs (a, b), a <= b < n_tiles); with slot (t, u) meaning "tile t's
// targets, from tile u":
//   * the square block t, u in [a0, a1): the action of (a, b) at (a, b) and its reaction at
//     (b, a), complementary triangles;
//   * actions of a band tile on the tiles b >= a1 after it, (a - a0) x (n_tiles - a1);
//   * reactions on those tiles, (b - a1) x (a - a0).
// One band covering every tile is the full square (n_tiles^2 slots).  Larger systems run several
// bands in turn, each reduced into float64 accumulators before the next, so the partial buffer
// is bounded by its first (largest) band while every sum keeps a fixed order.
struct SymSys {
    int64_t item0;            // first work item
    int64_t tile0;            // first (global) tile
    int64_t n_tiles, n_chunks;
    int64_t part0;            // first double of the system's partial block
    int64_t a0, a1;           // band of row tiles
    int shift0, n_img;        // image vectors shift0 .. shift0 + n_img - 1
    int n_g, img_per_g;       // image groups per tile pair and images per group
    int last_n;               // charges in the system's last chunk (1..kNearChunk; 0 = a full chunk)
    float tau2;               // coincident_r2 of the system's box (float32 kernels)
};
struct SymSysTable {
    SymSys one;
    const SymSys* many;       // nullptr: the launch has the single system `one`
    int n;
};

// tile pairs of the band: sum over a0 <= a < a1 of (n_tiles - a)
__host__ __device__ __forceinline__ int64_t sym_band_pairs(const SymSys& s) {
    const int64_t bw = s.a1 - s.a0;
    return bw * s.n_tiles - (s.a0 + s.a1 - 1) * bw / 2;
}
__host__ __device__ __forceinline__ int64_t sym_sys_items(const SymSys& s) {
    return sym_band_pairs(s) * s.n_g;
}
__host__ __device__ __forceinline__ int64_t sym_band_slots(const SymSys& s) {
    const int64_t bw = s.a1 - s.a0, n_out = s.n_tiles - s.a1;
    return bw * bw + 2 * bw * n_out;
}
__host__ __device__ __forceinline__ size_t sym_sys_doubles(const SymSys& s, int tile) {
    return (size_t)sym_band_slots(s) * (size_t)s.n_g * 4 * (size_t)tile;
}
// slot of tile t's targets for the contribution from tile u (see above)
__host__ __device__ __forceinline__ int64_t sym_slot(const SymSys& s, int64_t t, int64_t u) {
    const int64_t bw = s.a1 - s.a0, n_out = s.n_tiles - s.a1;
    if (t < s.a1) return u < s.a1 ? (t - s.a0) * bw + (u - s.a0) : bw * bw + (t - s.a0) * n_out + (u - s.a1);
    return bw * bw + bw * n_out + (t - s.a1) * bw + (u - s.a0);
}
// rows of the band's pairs before row a: sum over a0 <= a' < a of (n_tiles - a')
__host__ __device__ __forceinline__ int64_t sym_band_row_start(const SymSys& s, int64_t a) {
    const int64_t k = a - s.a0;
    return k * s.n_tiles - (s.a0 + a - 1) * k / 2;
}
// the band's pair with index p: row a (largest with row start <= p) and column b >= a
__host__ __device__ __forceinline__ void sym_band_pair(const SymSys& s, int64_t p, int64_t& a, int64_t& b) {
    int64_t lo = s.a0, hi = s.a1 - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (sym_band_row_start(s, mid) <= p) lo = mid; else hi = mid - 1;
    }
    a = lo;
    b = a + (p - sym_band_row_start(s, a));
}

struct NearSymLaunch {
    SymSysTable tab{};
    int64_t W = 0, G = 0;          // work items, resident CTAs
    int max_ipg = 0;               // largest images per group (shared-memory sizing)
    size_t doubles = 0;            // partial buffer
    int* counter = nullptr;
    int* status = nullptr;
    int n_status = 0;
    int inject = 0;
    int64_t debug_limit = 0;       // test hook of the debug bounds checks: a smaller partial buffer (doubles)
};

// Image groups: the fewest (1, 3, 9, ... up to one image per group) that give at least
// kSymItemsPerCta items per resident CTA over all systems, so that the last items finish
// close together.
#ifndef PSUM_SYM_ITEMS_PER_CTA
#define PSUM_SYM_ITEMS_PER_CTA 8
#endif
constexpr int kSymItemsPerCta = PSUM_SYM_ITEMS_PER_CTA;
// automatic choice (measured crossovers against the one-sided kernels): FP32C from 12 tiles of
// 512 charges (5500 charges even), float-float from 6 (3000 even), float64 at every size (1.64x
// at 1000 charges)
constexpr int64_t kSymMinTiles = 12;
constexpr int64_t kSymMinTilesFF = 6;
constexpr int64_t kSymMinTiles64 = 1;
constexpr size_t kSymMaxPartialBytes = (size_t)8 << 30;       // batches: a partial buffer of at most 8 GiB
// single systems: bands of row tiles whose partial slots fit this many bytes (one band up to
// 1.5 GiB: about 300 tiles of 512 charges in float32, 600 of 128 in float64)
#ifndef PSUM_SYM_BAND_BYTES
#define PSUM_SYM_BAND_BYTES ((size_t)3 << 29)
#endif
constexpr size_t kSymBandBytes = PSUM_SYM_BAND_BYTES;

// The widest equal band width whose first (largest) band -- bw^2 + 2 bw (n_tiles - bw) slots --
// fits `cap` bytes of slots of `slot_bytes` each; n_tiles when the whole square fits.
inline int64_t sym_band_width(int64_t n_tiles, size_t slot_bytes, size_t cap) {
    const int64_t cap_slots = (int64_t)(cap / (slot_bytes ? slot_bytes : 1));
    if (n_tiles * n_tiles <= cap_slots) return n_tiles;
    const double n = (double)n_tiles, c = (double)cap_slots;
    int64_t bw = (int64_t)(n - std::sqrt(n * n - c));
    if (bw < 1) bw = 1;
    while (bw > 1 && 2 * bw * n_tiles - bw * bw > cap_slots) --bw;
    while (bw + 1 < n_tiles && 2 * (bw + 1) * n_tiles - (bw + 1) * (bw + 1) <= cap_slots) ++bw;
    return bw;
}

// `sys` holds tile0, n_tiles, n_chunks, shift0 and n_img of every system; the rest is filled
// here.  G is the number of resident CTAs.
inline NearSymLaunch sym_partition(std::vector<SymSys>& sys, int64_t G, int tile = kTile32) {
    NearSymLaunch S;
    int64_t pairs = 0;
    int max_img = 1;
    for (const SymSys& s : sys) {
        pairs += s.n_tiles * (s.n_tiles + 1) / 2;
        max_img = s.n_img > max_img ? s.n_img : max_img;
    }
    int ng = 1;
    while (ng < max_img && pairs * ng < kSymItemsPerCta * G) ng *= 3;
    int64_t item = 0;
    size_t part = 0;
    for (SymSys& s : sys) {
        s.a0 = 0;
        s.a1 = s.n_tiles;
        const int g = ng < s.n_img ? ng : s.n_img;
        s.img_per_g = (s.n_img + g - 1) / g;
        s.n_g = (s.n_img + s.img_per_g - 1) / s.img_per_g;
        s.item0 = item;
        s.part0 = (int64_t)part;
        item += sym_sys_items(s);
        part += sym_sys_doubles(s, tile);
        S.max_ipg = s.img_per_g > S.max_ipg ? s.img_per_g : S.max_ipg;
    }
    S.W = item;
    S.doubles = part;
    S.G = G < S.W ? G : S.W;
    S.tab.one = sys.empty() ? SymSys{} : sys[0];
    S.tab.many = nullptr;
    S.tab.n = (int)sys.size();
    return S;
}

__device__ __forceinline__ int sym_sys_by_item(const SymSysTable& t, int64_t item) {
    if (!t.many) return 0;
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.many[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int sym_sys_by_tile(const SymSysTable& t, int64_t T) {
    if (!t.many) return 0;
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.many[mid].tile0 <= T) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Partition of the systems' units into work items for at most G_max resident CTAs; the partial
// buffer needs max_contrib slots per tile.  `dev_tab` is the device copy of `sys`
// (nullptr when there is one system).
inline NearPlanLaunch near_partition(const std::vector<NearSys>& sys, int64_t G_max, const NearSys* dev_tab,
                                     int items_per_cta = kItemsPerCta) {
    NearPlanLaunch L;
    L.U = 0;
    L.max_img = 1;
    L.n_tiles = 0;
    for (const NearSys& s : sys) {
        L.U += near_sys_units(s);
        L.max_img = s.n_img > L.max_img ? s.n_img : L.max_img;
        L.n_tiles = s.tile0 + s.n_tiles > L.n_tiles ? s.tile0 + s.n_tiles : L.n_tiles;
    }
    L.G = L.U < G_max ? L.U : G_max;
    if (L.G < 1) L.G = 1;
    // up to items_per_cta items per CTA, but items of at least kMinUnitsPerItem units where
    // the launch is small (every item adds a partial-sum slot to each tile it touches), and
    // at least one item per CTA
    L.W = L.G * (items_per_cta < 1 ? 1 : items_per_cta);
    if (L.W > L.U / kMinUnitsPerItem) L.W = L.U / kMinUnitsPerItem;
    if (L.W < L.G) L.W = L.G;
    if (L.W > L.U) L.W = L.U < 1 ? 1 : L.U;
    int mc = 1;
    for (const NearSys& s : sys) {
        const int64_t upt = s.n_chunks * s.n_img;
        for (int64_t t = 0; t < s.n_tiles; ++t) {
            const int64_t u0 = s.unit0 + t * upt;
            const int64_t g0 = sk_owner(u0, L.U, L.W);
            const int64_t g1 = sk_owner(u0 + upt - 1, L.U, L.W);
            if (g1 - g0 + 1 > mc) mc = (int)(g1 - g0 + 1);
        }
    }
    L.max_contrib = mc;
    L.tab.one = sys.empty() ? NearSys{} : sys[0];
    L.tab.many = sys.size() > 1 ? dev_tab : nullptr;
    L.tab.n = (int)sys.size();
    return L;
}

// The single-system case: targets tiles 0..n_tiles-1 against source chunks 0..n_chunks-1.
inline NearPlanLaunch near_partition(int64_t n_tiles, int64_t n_chunks, int n_img, int64_t G_max,
                                     int items_per_cta = kItemsPerCta) {
    std::vector<NearSys> one(1);
    one[0] = NearSys{0, 0, n_tiles, n_chunks, 0, 0, n_img, near_chunk_stride(n_chunks)};
    return near_partition(one, G_max, nullptr, items_per_cta);
}

}  // namespace psum

// The opaque plan handle of the C-ABI.
struct psum_plan_s {
    psum::Plan pl;
    int64_t launches = 0;       // kernels queued so far
    bool profile = false;
    bool inject_timeout = false;  // test hook: the charge pair kernel's copy waits run out
    int64_t debug_limit = 0;      // test hook: the partial buffers' size as the debug bounds checks see it
    int fail_allocs = 0;          // test hook: the next scratch allocations fail as if out of memory
    cudaEvent_t ev[6] = {};
    // the check-point sums and the box mean run on a side stream of the lowest priority, forked
    // after the packing and joined before the fit, so that they fill the SMs the persistent
    // charge kernel releases during its last work items
    cudaStream_t side = nullptr, side2 = nullptr;   // check sums; box mean
    cudaEvent_t fork0 = nullptr, fork = nullptr, join = nullptr, join2 = nullptr;
    // psum_eval_graph: one evaluation captured into a CUDA graph, replayed while the
    // arguments and the scratch buffer stay the same
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[6] = {};
    int64_t gN = 0;
    int64_t glaunches = 0;        // kernels one replay runs
};
