// Many independent periodic systems in one evaluation (psum_batch_*).
//
// Each system b has its own plan (box, degree, check points, near block) and a slice
// of the concatenated charges.  The charge pair sums of all systems form one unit space
// (cut into work items) and run as ONE persistent launch (the per-system table of the near
// kernels), and likewise the check-point pair sums; sorting, packing, validation, the
// least-squares fits, the means and the far fields run as one launch each, with a
// system descriptor per segment, group or block.  The whole sequence can be captured
// into a CUDA graph and replayed, and the pair-kernel variant is chosen by timing.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "launch.cuh"
#include "mean.cuh"

namespace psum {

constexpr int kSeg = 128;        // charges per segment (validation, mean, far field)
// systems of one batch: up to 256 sort with an 8-bit system prefix on the 24-bit Hilbert key
// (4 radix passes); more sort by the Hilbert key, then stably by the system (16 bits, 2 passes);
// per-system launches put the system in grid.y (at most 65535)
constexpr int kMaxBatch = 65535;
constexpr int kPrefixBatch = 256;

struct BatchDev {
    int64_t n0, n;            // the system's charges: rows n0 .. n0+n-1 (caller order = sorted order range)
    int64_t pt0;              // first packed charge point
    int64_t chk_pt0;          // first packed check point
    int64_t f0;               // first right-hand-side entry
    int64_t C0;               // first coefficient
    const double* pinv;       // (P-1) x M
    const double* Rbox;       // P
    const int* check_pos;     // 2M positions relative to chk_pt0, or M with `layers`
    const double* tab64;      // recurrence coefficients of the system's degree
    const float* tab32;
    int p, P, M, zero_mean;
    int layers;               // the check sums are the two-layer differences at the M points
    int seg0, nseg;
    double d[3], H[3];
    double inv_V0, inv_R0;
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// validation (Eq. 1), one block per segment of one system
__global__ void __launch_bounds__(kSeg) k_bvalidate(const double* __restrict__ x, const double* __restrict__ q,
                                                    const BatchDev* __restrict__ sys,
                                                    const int* __restrict__ seg_sys,
                                                    const int64_t* __restrict__ seg_start,
                                                    double* __restrict__ partial, int* __restrict__ status) {
    const int seg = blockIdx.x;
    const int b = seg_sys[seg];
    const BatchDev& S = sys[b];
    const int64_t i = seg_start[seg] + threadIdx.x;
    const bool valid = i < S.n0 + S.n;
    double s = 0.0, sa = 0.0;
    if (valid) {
        const double a = x[3 * i], c1 = x[3 * i + 1], c2 = x[3 * i + 2], qi = q[i];
        const bool in = (a >= -0.5 * S.d[0]) && (a < 0.5 * S.d[0]) && (c1 >= -0.5 * S.d[1]) &&
                        (c1 < 0.5 * S.d[1]) && (c2 >= -0.5 * S.d[2]) && (c2 < 0.5 * S.d[2]);
        int bad = in ? 0 : kStatOutOfBox;
        if (!(fabs(qi) <= 1.7976931348623157e308)) bad |= kStatNonFinite;
        if (bad) atomicOr(status + b, bad);
        s = qi;
        sa = fabs(qi);
    }
    __shared__ double ws[kSeg / 32], wa[kSeg / 32];
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        sa += __shfl_down_sync(0xffffffffu, sa, o);
    }
    if ((threadIdx.x & 31) == 0) { ws[threadIdx.x >> 5] = s; wa[threadIdx.x >> 5] = sa; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, ta = 0.0;
        for (int w = 0; w < kSeg / 32; ++w) { t += ws[w]; ta += wa[w]; }
        partial[2 * seg] = t;
        partial[2 * seg + 1] = ta;
    }
}

__global__ void k_bvalidate_finish(const BatchDev* __restrict__ sys, const double* __restrict__ partial,
                                   int* __restrict__ status) {
    const BatchDev& S = sys[blockIdx.x];
    double s = 0.0, sa = 0.0;
    for (int k = threadIdx.x; k < S.nseg; k += 32) {
        s += partial[2 * (S.seg0 + k)];
        sa += partial[2 * (S.seg0 + k) + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        sa += __shfl_down_sync(0xffffffffu, sa, o);
    }
    if (threadIdx.x == 0 && !(fabs(s) <= 1e-12 * sa)) atomicOr(status + blockIdx.x, kStatNonNeutral);
}

// sort keys: the 24-bit Hilbert index in the system's box, with the system in the top 8 bits
// when `prefix` (batches of up to 256 systems)
__global__ void __launch_bounds__(kSeg) k_bcurve_keys(const double* __restrict__ x, const BatchDev* __restrict__ sys,
                                                  const int* __restrict__ seg_sys,
                                                  const int64_t* __restrict__ seg_start, uint32_t* __restrict__ keys,
                                                  uint32_t* __restrict__ vals, int prefix) {
    const int seg = blockIdx.x;
    const int b = seg_sys[seg];
    const BatchDev& S = sys[b];
    const int64_t i = seg_start[seg] + threadIdx.x;
    if (i >= S.n0 + S.n) return;
    uint32_t c[3];
    for (int k = 0; k < 3; ++k) {
        const double u = (x[3 * i + k] / S.d[k] + 0.5) * 256.0;
        int v = (int)floor(u);
        v = v < 0 ? 0 : (v > 255 ? 255 : v);
        c[k] = (uint32_t)v;
    }
    keys[i] = (prefix ? (uint32_t)b << 24 : 0u) | hilbert_key24(c[0], c[1], c[2]);
    vals[i] = (uint32_t)i;
}

// after the curve-key passes of a large batch: the system of each sorted charge as the key of the
// remaining (stable) passes, found from its row by binary search over the systems' first rows
__global__ void k_bsys_keys(const uint32_t* __restrict__ vin, int64_t n, const BatchDev* __restrict__ sys, int B,
                            uint32_t* __restrict__ kout, uint32_t* __restrict__ vout) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t v = vin[j];
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sys[mid].n0 <= (int64_t)v) lo = mid; else hi = mid - 1;
    }
    kout[j] = (uint32_t)lo;
    vout[j] = v;
}

// step 4: f_l = phi_near(y~_l) - phi_near(y_l), for every system (grid.y = system); a
// system with two-layer check sums has the difference at y_l's position already
__global__ void k_brhs(const BatchDev* __restrict__ sys, const double* __restrict__ phi_check,
                       double* __restrict__ f) {
    const BatchDev& S = sys[blockIdx.y];
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= S.M) return;
    const double* pc = phi_check + S.chk_pt0;
    f[S.f0 + l] = S.layers ? pc[S.check_pos[l]] : pc[S.check_pos[S.M + l]] - pc[S.check_pos[l]];
}

// step 5: C_{2..P} = A^+ f, one warp per row (grid.y = system)
__global__ void __launch_bounds__(256) k_bproject(const BatchDev* __restrict__ sys, const double* __restrict__ f,
                                                  double* __restrict__ C) {
    const BatchDev& S = sys[blockIdx.y];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + w;
    if (row >= S.P - 1) return;
    const double* a = S.pinv + (int64_t)row * S.M;
    const double* fb = f + S.f0;
    double s = 0.0;
    for (int l = lane; l < S.M; l += 32) s = fma(a[l], fb[l], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) C[S.C0 + 1 + row] = s;
}

// mean of phi_near per segment (Eq. pfx4; the block potential by its regrouped corner sum)

__global__ void __launch_bounds__(kSeg) k_bbox_mean(const double* __restrict__ x, const double* __restrict__ q,
                                                    const BatchDev* __restrict__ sys,
                                                    const int* __restrict__ seg_sys,
                                                    const int64_t* __restrict__ seg_start,
                                                    double* __restrict__ partial) {
    const int seg = blockIdx.x;
    const BatchDev& S = sys[seg_sys[seg]];
    const int64_t i = seg_start[seg] + threadIdx.x;
    double s = 0.0;
    if (i < S.n0 + S.n && S.zero_mean) {
        const double X[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        s = q[i] * box_potential_paired(X, S.H);
    }
    __shared__ double ws[kSeg / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kSeg / 32; ++w) t += ws[w];
        partial[seg] = t;
    }
}

// step 6: C_1 = -<phi_near> - sum_{t>=2} C_t R_t^(0), one warp per system
__global__ void k_bconstant(const BatchDev* __restrict__ sys, const double* __restrict__ mean_partial,
                            double* __restrict__ C) {
    const BatchDev& S = sys[blockIdx.x];
    double s = 0.0, m = 0.0;
    if (S.zero_mean) {
        for (int t = 1 + threadIdx.x; t < S.P; t += 32) s = fma(C[S.C0 + t], S.Rbox[t], s);
        for (int k = threadIdx.x; k < S.nseg; k += 32) m += mean_partial[S.seg0 + k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        m += __shfl_down_sync(0xffffffffu, m, o);
    }
    if (threadIdx.x == 0) C[S.C0] = S.zero_mean ? (-m * S.inv_V0 - s) : 0.0;
}

// steps 7-8 per segment: phi = phi_near + phi_far, grad likewise, written in caller order
// (T = float for FP32C batches, double for FP64 and FF)
template <class T>
__global__ void __launch_bounds__(kSeg) k_bfar(const double* __restrict__ x, const BatchDev* __restrict__ sys,
                                               const int* __restrict__ seg_sys, const int64_t* __restrict__ seg_start,
                                               const uint32_t* __restrict__ perm, const double* __restrict__ phi_near,
                                               const double* __restrict__ grad_near, const double* __restrict__ C,
                                               int* __restrict__ status, double* __restrict__ phi,
                                               double* __restrict__ grad) {
    extern __shared__ unsigned char s_raw[];
    const int seg = blockIdx.x;
    const int b = seg_sys[seg];
    const BatchDev& S = sys[b];
    const int nt = sh_tab_size(S.p);
    T* s_C = (T*)s_raw;
    T* s_tab = s_C + S.P;
    const T* tab = sizeof(T) == sizeof(float) ? (const T*)S.tab32 : (const T*)S.tab64;
    for (int t = threadIdx.x; t < S.P; t += kSeg) s_C[t] = (T)C[S.C0 + t];
    for (int t = threadIdx.x; t < nt; t += kSeg) s_tab[t] = tab[t];
    __syncthreads();
    const int64_t s = seg_start[seg] + threadIdx.x;      // sorted position (caller position for FP64)
    if (s >= S.n0 + S.n) return;
    const int64_t i = perm ? (int64_t)perm[s] : s;
    const int64_t pk = S.pt0 + (s - S.n0);
    if (status[b] & (kStatNonNeutral | kStatOutOfBox | kStatNonFinite | kStatTimeout | kStatBounds)) {
        phi[i] = __longlong_as_double(0x7ff8000000000000ll);
        if (grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const T ux = (T)(x[3 * i] * S.inv_R0), uy = (T)(x[3 * i + 1] * S.inv_R0), uz = (T)(x[3 * i + 2] * S.inv_R0);
    T f = 0, gx = 0, gy = 0, gz = 0;
    if (grad) {
        sh_visit_tab<true>(ux, uy, uz, S.p, s_tab, [&](int nn, int mm, T v, T vx, T vy, T vz) {
            const T c = s_C[sh_index(nn, mm)];
            f = fma(c, v, f);
            gx = fma(c, vx, gx);
            gy = fma(c, vy, gy);
            gz = fma(c, vz, gz);
        });
    } else {
        sh_visit_tab<false>(ux, uy, uz, S.p, s_tab, [&](int nn, int mm, T v, T, T, T) {
            f = fma(s_C[sh_index(nn, mm)], v, f);
        });
    }
    const double ph = phi_near[pk] + (double)f;
    phi[i] = ph;
    bool finite = fabs(ph) <= 1.7976931348623157e308;
    if (grad) {
        const double g0 = grad_near[3 * pk] + (double)gx * S.inv_R0;
        const double g1 = grad_near[3 * pk + 1] + (double)gy * S.inv_R0;
        const double g2 = grad_near[3 * pk + 2] + (double)gz * S.inv_R0;
        grad[3 * i] = g0;
        grad[3 * i + 1] = g1;
        grad[3 * i + 2] = g2;
        finite = finite && fabs(g0) <= 1.7976931348623157e308 && fabs(g1) <= 1.7976931348623157e308 &&
                 fabs(g2) <= 1.7976931348623157e308;
    }
    if (!finite) atomicOr(status + b, kStatNonFinite);
}

}  // namespace psum

using namespace psum;

// ---------------------------------------------------------------------------
// the batch object
// ---------------------------------------------------------------------------
struct psum_batch_s {
    std::vector<psum_plan_t> plans;
    int B = 0, device = 0, precision = 0;
    int64_t N = 0;                      // charges
    int64_t n_pts = 0, n_chk_pts = 0;   // packed charge / check points
    int64_t n_groups = 0;               // packed charge groups
    int n_seg = 0;
    int max_P = 1;
    std::vector<BatchDev> sys;
    std::vector<NearSys> near_n, near_c;
    // device memory (one allocation)
    void* mem = nullptr;
    BatchDev* d_sys = nullptr;
    NearSys *d_near_n = nullptr, *d_near_c = nullptr;
    int* d_seg_sys = nullptr;
    int64_t* d_seg_start = nullptr;
    int64_t* d_grp_start = nullptr;
    int* d_grp_count = nullptr;
    double* d_shifts = nullptr;
    float4 *d_chk_hi = nullptr, *d_chk_lo = nullptr;
    double* d_chk_org = nullptr;
    // the check sums' image tables: per system its block images with weight 1, or, when the
    // batch runs the two-layer form (c_cls = kCheckClasses), its plan's two-layer tables for
    // its points' 6 classes (a system in the point form: class 0 its block images, the other
    // classes the same with weight 0); float32: the classes present in each check group
    int c_cls = 1;
    int* d_chk_cls = nullptr;
    double* d_chk_sub = nullptr;        // float32, two-layer form: [group][6][4] class spheres
    double* d_cshifts = nullptr;
    float* d_cw = nullptr;
    size_t n_centries = 0;
    double4_32a* d_chk64 = nullptr;
    uint32_t *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr, *hist = nullptr;
    float4 *pk_hi = nullptr, *pk_lo = nullptr;
    double* org = nullptr;
    float4* ext = nullptr;   // per group: bounding-box half extents (the symmetric kernel's near test)
    double4_32a* pk64 = nullptr;
    double *part_n = nullptr, *part_c = nullptr, *phi_n = nullptr, *grad_n = nullptr, *phi_c = nullptr;
    double *f = nullptr, *C = nullptr, *val_part = nullptr, *mean_part = nullptr;
    int* d_status = nullptr;
    int* h_status = nullptr;
    // schedule: variants 0 .. kNear32Variants - 1 are the one-sided charge kernel's register
    // budgets, variant kVariantSym the symmetric kernel (FP32C, partials within the cap)
    NearPlanLaunch Ln[kNear32Variants], Lc;
    std::vector<SymSys> sym_sys;
    SymSys* d_sym_sys = nullptr;
    NearSymLaunch Ls;
    bool sym_ok = false;
    double* part_s = nullptr;
    int variant = -1;
    double tuned_ms = 0.0;
    int64_t units = 0, pairs = 0;
    // graph
    cudaStream_t cap = nullptr;
    // the check-point sums, fits and means on a side stream of the lowest priority (forked after
    // the packing, joined before the constants): they fill the SMs the persistent charge kernel
    // releases during its last work items
    cudaStream_t side = nullptr, side2 = nullptr;   // check sums and fits; box means
    cudaEvent_t fork0 = nullptr, fork = nullptr, join = nullptr, join2 = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_args[5] = {};
    int64_t launches = 0;
};

namespace {

struct Bump2 {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += sizeof(T) * std::max<size_t>(count, 1);
        return p;
    }
};

int cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return PSUM_OK;
    if (e == cudaErrorMemoryAllocation) return PSUM_ERR_NOMEM;
    return PSUM_ERR_CUDA;
}

#define BTRY(expr)                                   \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) return cuda_st(e_);   \
    } while (0)

constexpr int kVariantSym = kNear32Variants;

// process-wide cache of autotuner decisions, keyed by the batch shape
std::mutex g_tune_mu;
std::map<std::pair<int64_t, int64_t>, int> g_tune_cache;

size_t batch_layout(psum_batch_s* bt, char* base) {
    Bump2 b{base};
    const bool fp32 = bt->precision != PSUM_FP64;   // float32 packing (FP32C and FF)
    const int B = bt->B;
    bt->d_sys = b.take<BatchDev>(B);
    bt->d_near_n = b.take<NearSys>(B);
    bt->d_near_c = b.take<NearSys>(B);
    bt->d_sym_sys = b.take<SymSys>(B);
    bt->d_seg_sys = b.take<int>(bt->n_seg);
    bt->d_seg_start = b.take<int64_t>(bt->n_seg);
    bt->d_grp_start = b.take<int64_t>(bt->n_groups);
    bt->d_grp_count = b.take<int>(bt->n_groups);
    size_t n_shift = 0;
    for (const psum_plan_t p : bt->plans) n_shift += 3 * (size_t)p->pl.n_images;
    bt->d_shifts = b.take<double>(n_shift);
    bt->d_chk_cls = b.take<int>((size_t)(bt->n_chk_pts / kNearChunk));
    bt->d_chk_sub = b.take<double>((size_t)(bt->n_chk_pts / kNearChunk) * kCheckClasses * 4);
    bt->d_cshifts = b.take<double>(3 * bt->n_centries);
    bt->d_cw = b.take<float>(bt->n_centries);
    if (fp32) {
        bt->d_chk_hi = b.take<float4>(2 * (size_t)bt->n_chk_pts);
        bt->d_chk_lo = b.take<float4>(2 * (size_t)bt->n_chk_pts);
        bt->d_chk_org = b.take<double>(4 * (size_t)(bt->n_chk_pts / kNearChunk));
        bt->ka = b.take<uint32_t>(bt->N);
        bt->va = b.take<uint32_t>(bt->N);
        bt->kb = b.take<uint32_t>(bt->N);
        bt->vb = b.take<uint32_t>(bt->N);
        bt->hist = b.take<uint32_t>((size_t)256 * sort_blocks(bt->N));
        bt->pk_hi = b.take<float4>(2 * (size_t)bt->n_pts);
        bt->pk_lo = b.take<float4>(2 * (size_t)bt->n_pts);
        bt->org = b.take<double>(4 * (size_t)bt->n_groups);
        bt->ext = b.take<float4>(bt->n_groups);
    } else {
        bt->d_chk64 = b.take<double4_32a>(bt->n_chk_pts);
        bt->pk64 = b.take<double4_32a>(bt->n_pts);
    }
    const int tile = fp32 ? kTile32 : kTile64;
    int mc_n = 1;
    for (int v = 0; v < (fp32 ? kNear32Variants : 1); ++v) mc_n = std::max(mc_n, bt->Ln[v].max_contrib);
    bt->part_n = b.take<double>((size_t)bt->Ln[0].n_tiles * mc_n * 4 * tile);
    bt->part_c = b.take<double>((size_t)bt->Lc.n_tiles * bt->Lc.max_contrib * tile);
    bt->part_s = bt->sym_ok ? b.take<double>(bt->Ls.doubles) : nullptr;
    bt->phi_n = b.take<double>(bt->n_pts);
    bt->grad_n = b.take<double>(3 * (size_t)bt->n_pts);
    bt->phi_c = b.take<double>(bt->n_chk_pts);
    int64_t nf = 0, nC = 0;
    for (const BatchDev& s : bt->sys) { nf += s.M; nC += s.P; }
    bt->f = b.take<double>(nf);
    bt->C = b.take<double>(nC);
    bt->val_part = b.take<double>(2 * (size_t)bt->n_seg);
    bt->mean_part = b.take<double>(bt->n_seg);
    bt->d_status = b.take<int>(B);
    int* counters = b.take<int>(2);            // work-item counters of the two pair launches
    for (int v = 0; v < kNear32Variants; ++v) bt->Ln[v].counter = counters;
    bt->Ls.counter = counters;
    bt->Lc.counter = counters + 1;
    for (int v = 0; v < kNear32Variants; ++v) {
        bt->Ln[v].status = bt->d_status;
        bt->Ln[v].n_status = B;
    }
    bt->Ls.status = bt->d_status;
    bt->Ls.n_status = B;
    bt->Lc.status = bt->d_status;
    bt->Lc.n_status = B;
    return b.off + 256;
}

int queue_batch(psum_batch_s* bt, const double* x, const double* q, double* phi, double* grad, cudaStream_t st,
                int variant) {
    const bool fp32 = bt->precision != PSUM_FP64;   // float32 packing (FP32C and FF)
    const int B = bt->B;
    int64_t nl = 0;
    // the box means need only the caller's charges: on the second side stream (least urgent
    // priority) from the start, where they fill the SMs that validation, sort and packing leave
    // idle, and the tail of the charge kernel
    BTRY(cudaEventRecord(bt->fork0, st));
    BTRY(cudaStreamWaitEvent(bt->side2, bt->fork0, 0));
    k_bbox_mean<<<bt->n_seg, kSeg, 0, bt->side2>>>(x, q, bt->d_sys, bt->d_seg_sys, bt->d_seg_start, bt->mean_part);
    BTRY(cudaEventRecord(bt->join2, bt->side2));
    BTRY(cudaMemsetAsync(bt->d_status, 0, sizeof(int) * B, st));
    k_bvalidate<<<bt->n_seg, kSeg, 0, st>>>(x, q, bt->d_sys, bt->d_seg_sys, bt->d_seg_start, bt->val_part,
                                            bt->d_status);
    k_bvalidate_finish<<<B, 32, 0, st>>>(bt->d_sys, bt->val_part, bt->d_status);
    nl += 2;
    const uint32_t* perm = nullptr;
    if (fp32) {
        const bool prefix = B <= kPrefixBatch;
        k_bcurve_keys<<<bt->n_seg, kSeg, 0, st>>>(x, bt->d_sys, bt->d_seg_sys, bt->d_seg_start, bt->ka, bt->va,
                                              prefix ? 1 : 0);
        if (prefix) {
            BTRY(launch_radix_sort(bt->ka, bt->va, bt->kb, bt->vb, bt->hist, bt->N, 4, st));
        } else {
            // curve-key passes (result in kb, vb), the systems as keys, two stable passes on them
            BTRY(launch_radix_sort(bt->ka, bt->va, bt->kb, bt->vb, bt->hist, bt->N, 3, st));
            k_bsys_keys<<<(unsigned)((bt->N + 255) / 256), 256, 0, st>>>(bt->vb, bt->N, bt->d_sys, B, bt->ka, bt->va);
            BTRY(launch_radix_sort(bt->ka, bt->va, bt->kb, bt->vb, bt->hist, bt->N, 2, st));
            nl += 1 + 6 - 3;
        }
        perm = bt->va;
        BTRY(launch_pack32_groups(x, q, perm, bt->n_groups, bt->d_grp_start, bt->d_grp_count, bt->pk_hi, bt->pk_lo,
                                  bt->org, st, bt->ext));
        nl += 1 + 12 + 1;
        const bool ff = bt->precision == PSUM_FF;
        BTRY(cudaEventRecord(bt->fork, st));
        if (variant == kVariantSym)
            BTRY(launch_near32s(bt->pk_hi, bt->pk_lo, bt->org, bt->ext, bt->d_shifts, bt->part_s, bt->Ls, st));
        else
            BTRY(launch_near32(true, bt->pk_hi, bt->pk_lo, bt->org, bt->pk_hi, bt->pk_lo, bt->org, bt->d_shifts,
                               bt->part_n, bt->Ln[variant], st, variant, nullptr, 0.0, ff));
        BTRY(cudaStreamWaitEvent(bt->side, bt->fork, 0));
        BTRY(launch_near32(false, bt->pk_hi, bt->pk_lo, bt->org, bt->d_chk_hi, bt->d_chk_lo, bt->d_chk_org,
                           bt->d_cshifts, bt->part_c, bt->Lc, bt->side, 0, nullptr, 0.0, ff, bt->d_chk_cls, bt->d_cw,
                           bt->c_cls, bt->d_chk_sub));
    } else {
        BTRY(launch_pack64_groups(x, q, bt->n_pts, bt->d_grp_start, bt->d_grp_count, bt->pk64, st));
        nl += 1;
        BTRY(cudaEventRecord(bt->fork, st));
        BTRY(launch_near64(true, bt->pk64, bt->pk64, bt->d_shifts, bt->part_n, bt->Ln[0], st));
        BTRY(cudaStreamWaitEvent(bt->side, bt->fork, 0));
        BTRY(launch_near64(false, bt->pk64, bt->d_chk64, bt->d_cshifts, bt->part_c, bt->Lc, bt->side, 0.0, bt->d_cw,
                           bt->c_cls));
    }
    // side stream: the check sums' reduction, the right-hand sides and the fits
    const int tile = fp32 ? kTile32 : kTile64;
    cudaStream_t sd = bt->side;
    BTRY(launch_near_reduce(bt->part_c, bt->n_chk_pts, tile, 1, bt->Lc, bt->phi_c, nullptr, sd));
    int maxM = 1, maxP = 1;
    for (const BatchDev& s : bt->sys) { maxM = std::max(maxM, s.M); maxP = std::max(maxP, s.P); }
    k_brhs<<<dim3((maxM + 255) / 256, B), 256, 0, sd>>>(bt->d_sys, bt->phi_c, bt->f);
    k_bproject<<<dim3((maxP - 1 + 7) / 8, B), 256, 0, sd>>>(bt->d_sys, bt->f, bt->C);
    BTRY(cudaEventRecord(bt->join, sd));
    if (variant == kVariantSym)
        BTRY(launch_sym_reduce(bt->part_s, bt->n_pts, bt->Ls, bt->phi_n, bt->grad_n, st));
    else
        BTRY(launch_near_reduce(bt->part_n, bt->n_pts, tile, 4, bt->Ln[fp32 ? variant : 0], bt->phi_n, bt->grad_n,
                                st));
    nl += 4;
    BTRY(cudaStreamWaitEvent(st, bt->join, 0));
    BTRY(cudaStreamWaitEvent(st, bt->join2, 0));
    k_bconstant<<<B, 32, 0, st>>>(bt->d_sys, bt->mean_part, bt->C);
    int max_tab = 1;
    for (const psum_plan_t p : bt->plans) max_tab = std::max(max_tab, sh_tab_size(p->pl.opt.p));
    if (bt->precision == PSUM_FP32C)
        k_bfar<float><<<bt->n_seg, kSeg, sizeof(float) * (maxP + max_tab), st>>>(
            x, bt->d_sys, bt->d_seg_sys, bt->d_seg_start, perm, bt->phi_n, grad ? bt->grad_n : nullptr, bt->C,
            bt->d_status, phi, grad);
    else
        k_bfar<double><<<bt->n_seg, kSeg, sizeof(double) * (maxP + max_tab), st>>>(
            x, bt->d_sys, bt->d_seg_sys, bt->d_seg_start, perm, bt->phi_n, grad ? bt->grad_n : nullptr, bt->C,
            bt->d_status, phi, grad);
    nl += 5;
    BTRY(cudaGetLastError());
    bt->launches += nl;
    return PSUM_OK;
}

// time the charge pair-sum variants on the current (packed) inputs and keep the fastest
int autotune(psum_batch_s* bt, cudaStream_t st) {
    // the plans' pair_kernel options: all PSUM_PAIRS_SYMMETRIC forces the symmetric kernel,
    // any PSUM_PAIRS_ONE_SIDED excludes it
    bool all_sym = true, any_one = false;
    for (const psum_plan_t p : bt->plans) {
        all_sym = all_sym && p->pl.opt.pair_kernel == PSUM_PAIRS_SYMMETRIC;
        any_one = any_one || p->pl.opt.pair_kernel == PSUM_PAIRS_ONE_SIDED;
    }
    const bool allow_sym = bt->sym_ok && !any_one;
    if (allow_sym && all_sym) {
        bt->variant = kVariantSym;
        return PSUM_OK;
    }
    const std::pair<int64_t, int64_t> key(bt->units,
                                          (int64_t)bt->precision * 1000 + bt->B + (allow_sym ? 1000000 : 0));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            bt->variant = it->second;
            return PSUM_OK;
        }
    }
    if (bt->precision != PSUM_FP32C) {
        bt->variant = 0;
        return PSUM_OK;
    }
    cudaEvent_t e0, e1;
    BTRY(cudaEventCreate(&e0));
    BTRY(cudaEventCreate(&e1));
    double best = 1e300;
    int best_v = 0;
    // each variant's charge pair kernel and its reduction (the symmetric kernel's reduction
    // reads more slots)
    for (int v = 0; v <= kVariantSym; ++v) {
        if (v == kVariantSym && !allow_sym) break;
        float ms = 0.f, tot = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            BTRY(cudaEventRecord(e0, st));
            if (v == kVariantSym) {
                BTRY(launch_near32s(bt->pk_hi, bt->pk_lo, bt->org, bt->ext, bt->d_shifts, bt->part_s, bt->Ls, st));
                BTRY(launch_sym_reduce(bt->part_s, bt->n_pts, bt->Ls, bt->phi_n, bt->grad_n, st));
            } else {
                BTRY(launch_near32(true, bt->pk_hi, bt->pk_lo, bt->org, bt->pk_hi, bt->pk_lo, bt->org, bt->d_shifts,
                                   bt->part_n, bt->Ln[v], st, v));
                BTRY(launch_near_reduce(bt->part_n, bt->n_pts, kTile32, 4, bt->Ln[v], bt->phi_n, bt->grad_n, st));
            }
            BTRY(cudaEventRecord(e1, st));
            BTRY(cudaEventSynchronize(e1));
            BTRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) tot += ms;          // the first launch of each variant warms up
        }
        bt->launches += 6;
        if (tot / 2 < best) {
            best = tot / 2;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bt->variant = best_v;
    bt->tuned_ms = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_v;
    return PSUM_OK;
}

class DevGuard {
   public:
    explicit DevGuard(int dev) {
        cudaGetDevice(&old_);
        if (old_ != dev) cudaSetDevice(dev);
    }
    ~DevGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != old_) cudaSetDevice(old_);
    }

   private:
    int old_ = 0;
};

void release(psum_batch_s* bt) {
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    if (bt->side) cudaStreamDestroy(bt->side);
    if (bt->side2) cudaStreamDestroy(bt->side2);
    if (bt->join2) cudaEventDestroy(bt->join2);
    if (bt->fork) cudaEventDestroy(bt->fork);
    if (bt->fork0) cudaEventDestroy(bt->fork0);
    if (bt->join) cudaEventDestroy(bt->join);
    cudaFree(bt->mem);
    if (bt->h_status) cudaFreeHost(bt->h_status);
}

}  // namespace

extern "C" {

int psum_batch_create(const psum_plan_t* plans, int B, const int64_t* offsets, psum_batch_t* out) {
    if (!plans || !offsets || !out || B < 1 || B > kMaxBatch || offsets[0] != 0) return PSUM_ERR_ARG;
    for (int b = 0; b < B; ++b) {
        if (!plans[b] || offsets[b + 1] <= offsets[b]) return PSUM_ERR_ARG;
        if (plans[b]->pl.opt.precision != plans[0]->pl.opt.precision) return PSUM_ERR_ARG;
        if (plans[b]->pl.device != plans[0]->pl.device) return PSUM_ERR_ARG;
        if (plans[b]->pl.Rb > 0.0) return PSUM_ERR_ARG;   // trimmed near sets: single-system path only
        if (plans[b]->pl.opt.basis != PSUM_BASIS_SPHERICAL) return PSUM_ERR_ARG;
    }
    if (offsets[B] > ((int64_t)1 << 30)) return PSUM_ERR_ARG;
    psum_batch_s* bt = new (std::nothrow) psum_batch_s();
    if (!bt) return PSUM_ERR_NOMEM;
    bt->plans.assign(plans, plans + B);
    bt->B = B;
    bt->device = plans[0]->pl.device;
    bt->precision = plans[0]->pl.opt.precision;
    bt->N = offsets[B];
    DevGuard dg(bt->device);
    const bool fp32 = bt->precision != PSUM_FP64;   // float32 packing (FP32C and FF)
    const bool ff = bt->precision == PSUM_FF;
    const int tile = fp32 ? kTile32 : kTile64;
    const int gpt = fp32 ? kTgt32 : 1;                  // groups (= chunks) per tile
    const int num_sms = plans[0]->pl.num_sms;

    // ---- per-system layout ----
    std::vector<int> seg_sys;
    std::vector<int64_t> seg_start, grp_start;
    std::vector<int> grp_count;
    int64_t pt = 0, chk_pt = 0, f0 = 0, C0 = 0, unit_n = 0, unit_c = 0, tile_n = 0, tile_c = 0;
    int shift0 = 0;
    int64_t cent0 = 0;                      // first entry of the system's check image table
    std::vector<int64_t> cent_first(B);
    // the two-layer form when a plan takes it and (float32) the per-class offsets of the
    // largest image list fit the kernel's shared memory
    {
        bool any = false;
        int max_c = 1;
        for (int b = 0; b < B; ++b) {
            const Plan& pl = plans[b]->pl;
            any = any || pl.lc_tiles > 0;
            max_c = std::max(max_c, pl.lc_tiles > 0 ? pl.lc_img : pl.n_images);
        }
        bt->c_cls = any && (!fp32 || near32_dyn_smem(max_c, false, false, kCheckClasses) <= kNear32DynSmemMax)
                        ? kCheckClasses : 1;
    }
    bt->sys.resize(B);
    bt->near_n.resize(B);
    bt->near_c.resize(B);
    bt->sym_sys.resize(B);
    for (int b = 0; b < B; ++b) {
        const Plan& pl = plans[b]->pl;
        const int64_t n = offsets[b + 1] - offsets[b];
        const int64_t n_tiles = (n + tile - 1) / tile;
        const int64_t n_chunks = (n + kNearChunk - 1) / kNearChunk;
        BatchDev& S = bt->sys[b];
        S.n0 = offsets[b];
        S.n = n;
        S.pt0 = pt;
        S.chk_pt0 = chk_pt;
        S.f0 = f0;
        S.C0 = C0;
        S.pinv = pl.d_pinv;
        S.Rbox = pl.d_Rbox;
        // plans with two-layer tables keep that form in the batch
        const bool layers = bt->c_cls > 1 && pl.lc_tiles > 0;
        S.layers = layers ? 1 : 0;
        S.check_pos = layers ? pl.d_lc_pos : pl.d_check_pos;
        S.tab64 = pl.d_shtab64;
        S.tab32 = pl.d_shtab32;
        S.p = pl.opt.p;
        S.P = pl.P;
        S.M = pl.opt.M;
        S.zero_mean = pl.opt.mean_mode == PSUM_MEAN_ZERO;
        S.seg0 = (int)seg_sys.size();
        S.nseg = (int)((n + kSeg - 1) / kSeg);
        for (int k = 0; k < 3; ++k) {
            S.d[k] = pl.opt.d[k];
            S.H[k] = 0.5 * (2 * pl.opt.K[k] + 1) * pl.opt.d[k];
        }
        S.inv_V0 = 1.0 / (pl.opt.d[0] * pl.opt.d[1] * pl.opt.d[2]);
        S.inv_R0 = 1.0 / pl.R0;
        for (int k = 0; k < S.nseg; ++k) {
            seg_sys.push_back(b);
            seg_start.push_back(S.n0 + (int64_t)k * kSeg);
        }
        for (int64_t g = 0; g < n_tiles * gpt; ++g) {
            grp_start.push_back(S.n0 + g * kNearChunk);
            grp_count.push_back((int)std::max<int64_t>(0, std::min<int64_t>(kNearChunk, n - g * kNearChunk)));
        }
        const int64_t chk_tiles = layers ? pl.lc_tiles : pl.n_check_tiles;
        const int c_img = layers ? pl.lc_img : pl.n_images;
        bt->near_n[b] = NearSys{unit_n, tile_n, n_tiles, n_chunks, pt / kNearChunk, shift0, pl.n_images,
                                near_chunk_stride(n_chunks), coincident_r2(pl.opt.d)};
        // the check sums index their own image tables (cent0)
        bt->near_c[b] = NearSys{unit_c, tile_c, chk_tiles, n_chunks, pt / kNearChunk, (int)cent0, c_img,
                                near_chunk_stride(n_chunks), coincident_r2(pl.opt.d)};
        cent_first[b] = cent0;
        cent0 += (int64_t)bt->c_cls * c_img;
        SymSys ss{};
        ss.tile0 = tile_n;
        ss.n_tiles = n_tiles;
        ss.n_chunks = n_chunks;
        ss.last_n = n_chunks > 0 ? (int)(n - (n_chunks - 1) * kNearChunk) : 0;
        ss.tau2 = coincident_r2(pl.opt.d);
        ss.shift0 = shift0;
        ss.n_img = pl.n_images;
        bt->sym_sys[b] = ss;
        unit_n += near_sys_units(bt->near_n[b]);
        unit_c += near_sys_units(bt->near_c[b]);
        tile_n += n_tiles;
        tile_c += chk_tiles;
        pt += n_tiles * tile;
        chk_pt += chk_tiles * tile;
        f0 += S.M;
        C0 += S.P;
        shift0 += pl.n_images;
        bt->max_P = std::max(bt->max_P, S.P);
        bt->pairs += (int64_t)pl.n_images * n * (n + 2 * S.M);
    }
    bt->n_pts = pt;
    bt->n_chk_pts = chk_pt;
    bt->n_centries = (size_t)cent0;
    bt->n_groups = pt / kNearChunk;
    bt->n_seg = (int)seg_sys.size();
    bt->units = unit_n;

    // schedules: one work-item partition per pair-kernel variant for the charges, one for the
    // check points; the device tables they point to are filled below
    int max_img = 1;
    for (int b = 0; b < B; ++b) max_img = std::max(max_img, plans[b]->pl.n_images);
    for (int v = 0; v < (fp32 ? kNear32Variants : 1); ++v) {
        const int64_t gmax = (int64_t)num_sms * (fp32 ? near32_occupancy_ctas(max_img, v, false, ff)
                                                       : near64_occupancy_ctas());
        bt->Ln[v] = near_partition(bt->near_n, gmax, nullptr);
    }
    {
        const int64_t gmax = (int64_t)num_sms * (fp32 ? near32_occupancy_ctas(max_img, 0, false, ff)
                                                       : near64_occupancy_ctas());
        bt->Lc = near_partition(bt->near_c, gmax, nullptr, kCheckItemsPerCta);
    }
    if (bt->precision == PSUM_FP32C) {
        bt->Ls = sym_partition(bt->sym_sys, (int64_t)num_sms * near32s_occupancy_ctas(max_img, false));
        bt->Ls.G = std::min<int64_t>((int64_t)num_sms * near32s_occupancy_ctas(bt->Ls.max_ipg, false), bt->Ls.W);
        bt->sym_ok = bt->Ls.W > 0 && bt->Ls.doubles * sizeof(double) <= kSymMaxPartialBytes;
    }
    int st = PSUM_OK;
    const size_t bytes = batch_layout(bt, nullptr);
    cudaError_t e = cudaMalloc(&bt->mem, bytes);
    if (e != cudaSuccess) {
        delete bt;
        return cuda_st(e);
    }
    batch_layout(bt, (char*)bt->mem);
    if (B > 1) {
        for (int v = 0; v < kNear32Variants; ++v) bt->Ln[v].tab.many = bt->d_near_n;
        bt->Lc.tab.many = bt->d_near_c;
        bt->Ls.tab.many = bt->d_sym_sys;
    }
    // ---- upload tables and concatenate the plans' check targets and image vectors ----
    auto up = [&](void* dst, const void* src, size_t n) -> int {
        if (n == 0) return PSUM_OK;
        return cuda_st(cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice));
    };
    if ((st = up(bt->d_sys, bt->sys.data(), sizeof(BatchDev) * B)) ||
        (st = up(bt->d_near_n, bt->near_n.data(), sizeof(NearSys) * B)) ||
        (st = up(bt->d_near_c, bt->near_c.data(), sizeof(NearSys) * B)) ||
        (st = up(bt->d_sym_sys, bt->sym_sys.data(), sizeof(SymSys) * B)) ||
        (st = up(bt->d_seg_sys, seg_sys.data(), sizeof(int) * seg_sys.size())) ||
        (st = up(bt->d_seg_start, seg_start.data(), sizeof(int64_t) * seg_start.size())) ||
        (st = up(bt->d_grp_start, grp_start.data(), sizeof(int64_t) * grp_start.size())) ||
        (st = up(bt->d_grp_count, grp_count.data(), sizeof(int) * grp_count.size()))) {
        release(bt);
        delete bt;
        return st;
    }
    size_t so = 0;
    for (int b = 0; b < B && st == PSUM_OK; ++b) {
        const Plan& pl = plans[b]->pl;
        st = cuda_st(cudaMemcpy(bt->d_shifts + so, pl.d_shifts, sizeof(double) * 3 * pl.n_images,
                                cudaMemcpyDeviceToDevice));
        so += 3 * (size_t)pl.n_images;
        const BatchDev& S = bt->sys[b];
        const size_t npts = (size_t)(S.layers ? pl.lc_tiles : pl.n_check_tiles) * tile;
        const size_t ngrp = npts / kNearChunk;
        if (st == PSUM_OK && fp32) {
            const float4* src = (const float4*)(S.layers ? pl.d_lc_tgt : pl.d_check_tgt);
            const double* corg = S.layers ? pl.d_lc_org : pl.d_check_org;
            st = cuda_st(cudaMemcpy(bt->d_chk_hi + 2 * S.chk_pt0, src, sizeof(float4) * 2 * npts,
                                    cudaMemcpyDeviceToDevice));
            if (st == PSUM_OK)
                st = cuda_st(cudaMemcpy(bt->d_chk_lo + 2 * S.chk_pt0, src + 2 * npts, sizeof(float4) * 2 * npts,
                                        cudaMemcpyDeviceToDevice));
            if (st == PSUM_OK)
                st = cuda_st(cudaMemcpy(bt->d_chk_org + 4 * (S.chk_pt0 / kNearChunk), corg,
                                        sizeof(double) * 4 * ngrp, cudaMemcpyDeviceToDevice));
        } else if (st == PSUM_OK) {
            st = cuda_st(cudaMemcpy(bt->d_chk64 + S.chk_pt0, S.layers ? pl.d_lc_tgt : pl.d_check_tgt,
                                    sizeof(double4_32a) * npts, cudaMemcpyDeviceToDevice));
        }
        // the system's check image table and group classes
        const size_t ce = (size_t)cent_first[b];
        if (st == PSUM_OK && S.layers) {
            const size_t n_e = (size_t)kCheckClasses * pl.lc_img;
            st = cuda_st(cudaMemcpy(bt->d_cshifts + 3 * ce, pl.d_lc_shifts, sizeof(double) * 3 * n_e,
                                    cudaMemcpyDeviceToDevice));
            if (st == PSUM_OK)
                st = cuda_st(cudaMemcpy(bt->d_cw + ce, pl.d_lc_w, sizeof(float) * n_e, cudaMemcpyDeviceToDevice));
            if (st == PSUM_OK && fp32)
                st = cuda_st(cudaMemcpy(bt->d_chk_cls + S.chk_pt0 / kNearChunk, pl.d_lc_gmask, sizeof(int) * ngrp,
                                        cudaMemcpyDeviceToDevice));
            if (st == PSUM_OK && fp32)
                st = cuda_st(cudaMemcpy(bt->d_chk_sub + (S.chk_pt0 / kNearChunk) * kCheckClasses * 4, pl.d_lc_sub,
                                        sizeof(double) * ngrp * kCheckClasses * 4, cudaMemcpyDeviceToDevice));
        } else if (st == PSUM_OK) {
            // the block images for every class (weight 1 for class 0, which all its points have)
            std::vector<float> wts((size_t)bt->c_cls * pl.n_images, 0.f);
            std::fill(wts.begin(), wts.begin() + pl.n_images, 1.f);
            for (int c = 0; c < bt->c_cls && st == PSUM_OK; ++c)
                st = cuda_st(cudaMemcpy(bt->d_cshifts + 3 * (ce + (size_t)c * pl.n_images), pl.d_shifts,
                                        sizeof(double) * 3 * pl.n_images, cudaMemcpyDeviceToDevice));
            if (st == PSUM_OK)
                st = cuda_st(cudaMemcpy(bt->d_cw + ce, wts.data(), sizeof(float) * wts.size(), cudaMemcpyHostToDevice));
            if (st == PSUM_OK && fp32) {
                const std::vector<int> ones(ngrp, 1);
                st = cuda_st(cudaMemcpy(bt->d_chk_cls + S.chk_pt0 / kNearChunk, ones.data(), sizeof(int) * ngrp,
                                        cudaMemcpyHostToDevice));
                // every class's sphere is the group's own (only class 0 occurs)
                std::vector<double> org(4 * ngrp), sub(ngrp * kCheckClasses * 4);
                if (st == PSUM_OK)
                    st = cuda_st(cudaMemcpy(org.data(), pl.d_check_org, sizeof(double) * org.size(),
                                            cudaMemcpyDeviceToHost));
                for (size_t g = 0; g < ngrp; ++g)
                    for (int c = 0; c < kCheckClasses; ++c)
                        for (int k = 0; k < 4; ++k) sub[4 * (g * kCheckClasses + c) + k] = org[4 * g + k];
                if (st == PSUM_OK)
                    st = cuda_st(cudaMemcpy(bt->d_chk_sub + (S.chk_pt0 / kNearChunk) * kCheckClasses * 4, sub.data(),
                                            sizeof(double) * sub.size(), cudaMemcpyHostToDevice));
            }
        }
    }
    if (st == PSUM_OK) st = cuda_st(cudaMallocHost((void**)&bt->h_status, sizeof(int) * B));
    if (st == PSUM_OK) st = cuda_st(cudaMemset(bt->d_status, 0, sizeof(int) * B));
    if (st == PSUM_OK) st = cuda_st(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
    if (st == PSUM_OK) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        st = cuda_st(cudaStreamCreateWithPriority(&bt->side, cudaStreamNonBlocking, lo));
        if (st == PSUM_OK) st = cuda_st(cudaStreamCreateWithPriority(&bt->side2, cudaStreamNonBlocking, lo));
    }
    if (st == PSUM_OK) st = cuda_st(cudaEventCreateWithFlags(&bt->join2, cudaEventDisableTiming));
    if (st == PSUM_OK) st = cuda_st(cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming));
    if (st == PSUM_OK) st = cuda_st(cudaEventCreateWithFlags(&bt->fork0, cudaEventDisableTiming));
    if (st == PSUM_OK) st = cuda_st(cudaEventCreateWithFlags(&bt->join, cudaEventDisableTiming));
    if (st != PSUM_OK) {
        release(bt);
        delete bt;
        return st;
    }
    *out = bt;
    return PSUM_OK;
}

int psum_batch_eval(psum_batch_t bt, const double* x, const double* q, double* phi, double* grad, int use_graph,
                    void* stream) {
    if (!bt || !x || !q || !phi) return PSUM_ERR_ARG;
    DevGuard dg(bt->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (bt->variant < 0) {
        // first evaluation: run it plainly, then time the variants on its packed inputs; the
        // outputs come from the chosen variant (the symmetric kernel rounds differently)
        int s = queue_batch(bt, x, q, phi, grad, st, 0);
        if (s != PSUM_OK) return s;
        s = autotune(bt, st);
        if (s != PSUM_OK) return s;
        if (!use_graph && bt->variant == 0) return PSUM_OK;
    }
    if (!use_graph) return queue_batch(bt, x, q, phi, grad, st, bt->variant);
    const void* args[5] = {x, q, phi, grad, stream};
    bool same = bt->exec != nullptr;
    for (int k = 0; k < 5 && same; ++k) same = bt->g_args[k] == args[k];
    if (!same) {
        if (bt->exec) {
            cudaGraphExecDestroy(bt->exec);
            bt->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        BTRY(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
        const int64_t before = bt->launches;
        const int s = queue_batch(bt, x, q, phi, grad, bt->cap, bt->variant);
        const cudaError_t e = cudaStreamEndCapture(bt->cap, &graph);
        bt->launches = before;                     // capturing queues nothing on the device
        if (s != PSUM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        BTRY(e);
        const cudaError_t ei = cudaGraphInstantiate(&bt->exec, graph, 0);
        cudaGraphDestroy(graph);
        BTRY(ei);
        for (int k = 0; k < 5; ++k) bt->g_args[k] = args[k];
    }
    BTRY(cudaGraphLaunch(bt->exec, st));
    bt->launches += 2 + (bt->precision != PSUM_FP64 ? 14 : 1) + 4 + 5;
    return PSUM_OK;
}

int psum_batch_sync(psum_batch_t bt, int* status, void* stream) {
    if (!bt) return PSUM_ERR_ARG;
    DevGuard dg(bt->device);
    cudaStream_t st = (cudaStream_t)stream;
    BTRY(cudaMemcpyAsync(bt->h_status, bt->d_status, sizeof(int) * bt->B, cudaMemcpyDeviceToHost, st));
    BTRY(cudaMemsetAsync(bt->d_status, 0, sizeof(int) * bt->B, st));
    BTRY(cudaStreamSynchronize(st));
    int first = PSUM_OK;
    for (int b = 0; b < bt->B; ++b) {
        const int s = bt->h_status[b];
        int code = PSUM_OK;
        if (s & kStatBounds) code = PSUM_ERR_INTERNAL;
        else if (s & kStatNonNeutral) code = PSUM_ERR_NONNEUTRAL;
        else if (s & kStatOutOfBox) code = PSUM_ERR_OUT_OF_BOX;
        else if (s & kStatNonFinite) code = PSUM_ERR_NONFINITE;
        else if (s & kStatTimeout) code = PSUM_ERR_TIMEOUT;
        if (status) status[b] = code;
        if (first == PSUM_OK) first = code;
    }
    return first;
}

int psum_batch_get_coeffs(psum_batch_t bt, int b, double* C, void* stream) {
    if (!bt || !C || b < 0 || b >= bt->B) return PSUM_ERR_ARG;
    DevGuard dg(bt->device);
    cudaStream_t st = (cudaStream_t)stream;
    BTRY(cudaMemcpyAsync(C, bt->C + bt->sys[b].C0, sizeof(double) * bt->sys[b].P, cudaMemcpyDeviceToHost, st));
    BTRY(cudaStreamSynchronize(st));
    return PSUM_OK;
}

int psum_batch_get_info(psum_batch_t bt, psum_batch_info* info) {
    if (!bt || !info) return PSUM_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->B = bt->B;
    info->N_total = bt->N;
    info->units = bt->units;
    info->pairs = bt->pairs;
    const int v = bt->variant < 0 ? 0 : bt->variant;
    info->ctas = (int)(v == kVariantSym ? bt->Ls.G : bt->Ln[v].G);
    info->variant = bt->variant;
    info->tuned_ms = bt->tuned_ms;
    return PSUM_OK;
}

void psum_batch_destroy(psum_batch_t bt) {
    if (!bt) return;
    {
        DevGuard dg(bt->device);
        cudaDeviceSynchronize();
        release(bt);
    }
    delete bt;
}

}  // extern "C"
