// C-ABI entry points (include/psum.h) and the device pipeline of algorithm
// "get" (Sec. 2.3.2), queued on the caller's stream.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "psum_internal.cuh"

#include "launch.cuh"

using namespace psum;


namespace {

struct Bump {
    char* base;
    size_t off = 0;
    size_t cap;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += sizeof(T) * std::max<size_t>(count, 1);
        return p;
    }
};

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PSUM_OK;
    if (e == cudaErrorMemoryAllocation) return PSUM_ERR_NOMEM;
    return PSUM_ERR_CUDA;
}

// register budget of the check sums (the 6-CTA instance exists for untrimmed FP32C plans only)
int check_variant(const Plan& pl) {
    return pl.opt.precision == PSUM_FP32C && !(pl.Rb > 0.0) ? kCheckVariant : 0;
}

// refined float32 pair terms (PSUM_TERMS_REFINED) in the symmetric charge kernel of FP32C plans
bool refined_terms(const Plan& pl) {
    return pl.opt.precision == PSUM_FP32C && pl.opt.fp32_terms == PSUM_TERMS_REFINED;
}

int map_device_status(int s) {
    if (s & kStatBounds) return PSUM_ERR_INTERNAL;
    if (s & kStatNonNeutral) return PSUM_ERR_NONNEUTRAL;
    if (s & kStatOutOfBox) return PSUM_ERR_OUT_OF_BOX;
    if (s & kStatNonFinite) return PSUM_ERR_NONFINITE;
    if (s & kStatTimeout) return PSUM_ERR_TIMEOUT;
    return PSUM_OK;
}

__global__ void k_status_merge(const int* eval_status, int* plan_status) {
    if (*eval_status) atomicOr(plan_status, *eval_status);
}

struct Layout {
    // FP32C
    uint32_t *ka, *va, *kb, *vb, *hist;
    float4 *pk32, *pk32lo;
    double* org;
    float4* ext;         // per charge group: bounding-box half extents (the symmetric kernel's near test)
    double* xs;          // float64 packed source positions (trimmed plans)
    // FP64
    double4_32a* pk64;
    // common
    double *part_n, *part_c, *phi_n, *grad_n, *phi_c, *val_part, *mean_part, *f;
    int* eval_status;
    // backward
    double *far_phi, *far_grad, *w_part, *w, *u, *psi, *gpsi, *part_b;
    float4* chk_src32;
    float4* chk_src32lo;   // float-float plans: lo parts of the check points as sources
    double4_32a* chk_src64;
    NearPlanLaunch Lb;
    int nblk_mom;
    NearPlanLaunch Ln, Lc;
    bool sym;              // the charge pair sums by the symmetric kernel (partition S)
    NearSymLaunch S;       // its first band (row tiles 0 .. sym_bw - 1)
    int64_t sym_bw = 0, sym_bands = 0;   // band width (row tiles) and number of bands
    int64_t n_tiles, n_chunks, n_pts;   // target tiles, source chunks, packed target points
    int64_t n_src_groups, n_src_pts;    // the charges' pack (groups of 128, FP32C/FF; points, FP64)
    int nblk_val, nblk_mean;
    // separate evaluation points (psum_eval_points): their sort and pack; null otherwise
    uint32_t *tka, *tva, *tkb, *tvb, *thist;
    float4 *tpk32, *tpk32lo;
    double* torg;
    double4_32a* tpk64;
};

// Split the single system of L.S (one full band) into bands of row tiles whose partial slots
// fit `cap` bytes (kSymBandBytes unless a test lowers it); L.S becomes the first band.
void sym_bands(Layout& L, int tile, size_t cap) {
    SymSys& s = L.S.tab.one;
    const int64_t G = L.S.G;
    L.sym_bw = sym_band_width(s.n_tiles, (size_t)s.n_g * 4 * tile * sizeof(double), cap ? cap : kSymBandBytes);
    L.sym_bands = (s.n_tiles + L.sym_bw - 1) / L.sym_bw;
    s.a0 = 0;
    s.a1 = L.sym_bw;
    s.item0 = 0;
    L.S.W = sym_sys_items(s);
    L.S.doubles = sym_sys_doubles(s, tile);
    L.S.G = G < L.S.W ? G : L.S.W;
}

// The launch of band k of the symmetric partition (row tiles k bw .. (k + 1) bw - 1).
NearSymLaunch sym_band_launch(const Layout& L, int64_t k, bool inject, int64_t debug_limit = 0) {
    NearSymLaunch S = L.S;
    S.debug_limit = debug_limit;
    SymSys& b = S.tab.one;
    b.a0 = k * L.sym_bw;
    b.a1 = std::min(b.n_tiles, b.a0 + L.sym_bw);
    S.W = sym_sys_items(b);
    S.G = std::min(L.S.G, S.W);
    S.inject = inject ? 1 : 0;
    return S;
}

// Lay out the scratch buffer for N charges; with base == nullptr only the size is computed.
// `backward` adds the buffers of the energy derivatives; T >= 0 adds T separate evaluation
// points (their sort and pack), T < 0 evaluates at the charges.
size_t layout(Plan& pl, int64_t N, char* base, Layout& L, bool backward = false, int64_t g_cap = 0,
              int64_t T = -1) {
    Bump b{base, 0, 0};
    const bool sep = T >= 0;
    const int64_t NT = sep ? T : N;            // evaluation points
    const bool fp32 = pl.opt.precision != PSUM_FP64;   // float32 packing (FP32C and FF)
    const int n_img = pl.n_images;
    // a capped width (the allocation-free entry) keeps one work item per CTA: the partial
    // sums grow with the number of items
    const int ipc = g_cap > 0 ? 1 : kItemsPerCta;
    L.tka = L.tva = L.tkb = L.tvb = L.thist = nullptr;
    L.tpk32 = L.tpk32lo = nullptr;
    L.torg = nullptr;
    L.tpk64 = nullptr;
    if (fp32) {
        L.n_tiles = (NT + kTile32 - 1) / kTile32;
        L.n_chunks = (N + kNearChunk - 1) / kNearChunk;
        const int64_t n_groups = L.n_tiles * kTgt32;
        L.n_pts = n_groups * kNearChunk;
        L.n_src_groups = sep ? L.n_chunks : n_groups;
        L.n_src_pts = L.n_src_groups * kNearChunk;
        const bool trimmed = pl.Rb > 0.0;
        const bool ffp0 = pl.opt.precision == PSUM_FF;
        int64_t gmax = (int64_t)pl.num_sms * near32_occupancy_ctas(n_img, 0, trimmed, ffp0);
        if (g_cap > 0 && gmax > g_cap) gmax = g_cap;
        L.Ln = near_partition(L.n_tiles, L.n_chunks, n_img, gmax, ipc);
        L.Ln.tab.one.tau2 = coincident_r2(pl.opt.d);
        // check sums: the 2M points with the block's images, or the M points with their
        // class's two image layers
        const bool layers = pl.lc_tiles > 0;
        const int64_t c_tiles = layers ? pl.lc_tiles : pl.n_check_tiles;
        // the check sums' own instance (potential only) sets their width
        const int cv = check_variant(pl);
        int64_t gmax_c = (int64_t)pl.num_sms * near32_occupancy_ctas(layers ? pl.lc_img : n_img, cv, trimmed, ffp0, false,
                                                                      layers ? kCheckClasses : 1);
        if (g_cap > 0 && gmax_c > g_cap) gmax_c = g_cap;
        L.Lc = near_partition(c_tiles, L.n_chunks, layers ? pl.lc_img : n_img, gmax_c,
                              g_cap > 0 ? 1 : kCheckItemsPerCta);
        L.Lc.tab.one.tau2 = coincident_r2(pl.opt.d);
        // the symmetric kernel: FP32C charges, block image set, a normal (growing) scratch
        L.sym = false;
        const int pk = pl.opt.pair_kernel;
        const bool ffp = pl.opt.precision == PSUM_FF;
        if (!sep && !trimmed && g_cap == 0 && pk != PSUM_PAIRS_ONE_SIDED &&
            (pk == PSUM_PAIRS_SYMMETRIC || L.n_tiles >= (ffp ? kSymMinTilesFF : kSymMinTiles))) {
            // image groups sized for the occupancy of the largest group (the largest dynamic
            // shared memory), then the launch width for the chosen group size
            std::vector<SymSys> one(1);
            one[0].tile0 = 0;
            one[0].n_tiles = L.n_tiles;
            one[0].n_chunks = L.n_chunks;
            one[0].last_n = (int)(N - (L.n_chunks - 1) * kNearChunk);
            one[0].shift0 = 0;
            one[0].n_img = n_img;
            one[0].tau2 = coincident_r2(pl.opt.d);
            const bool rf = refined_terms(pl);
            L.S = sym_partition(one, (int64_t)pl.num_sms * near32s_occupancy_ctas(n_img, ffp, rf));
            L.S.G = (int64_t)pl.num_sms * near32s_occupancy_ctas(L.S.max_ipg, ffp, rf);
            sym_bands(L, kTile32, pl.sym_band_bytes);
            L.sym = true;
        }
        L.xs = trimmed ? b.take<double>(3 * (size_t)L.n_src_pts) : nullptr;
        L.ka = b.take<uint32_t>(N);
        L.va = b.take<uint32_t>(N);
        L.kb = b.take<uint32_t>(N);
        L.vb = b.take<uint32_t>(N);
        L.hist = b.take<uint32_t>((size_t)256 * sort_blocks(N));
        L.pk32 = b.take<float4>(2 * (size_t)L.n_src_pts);
        L.pk32lo = b.take<float4>(2 * (size_t)L.n_src_pts);
        L.org = b.take<double>(4 * (size_t)L.n_src_groups);
        L.ext = L.sym ? b.take<float4>(L.n_src_groups) : nullptr;
        L.pk64 = nullptr;
        if (sep) {
            L.tka = b.take<uint32_t>(T);
            L.tva = b.take<uint32_t>(T);
            L.tkb = b.take<uint32_t>(T);
            L.tvb = b.take<uint32_t>(T);
            L.thist = b.take<uint32_t>((size_t)256 * sort_blocks(T));
            L.tpk32 = b.take<float4>(2 * (size_t)L.n_pts);
            L.tpk32lo = b.take<float4>(2 * (size_t)L.n_pts);
            L.torg = b.take<double>(4 * (size_t)n_groups);
        }
        L.part_n = b.take<double>(L.sym ? L.S.doubles : (size_t)L.n_tiles * L.Ln.max_contrib * 4 * kTile32);
        L.part_c = b.take<double>((size_t)c_tiles * L.Lc.max_contrib * kTile32);
        L.phi_c = b.take<double>((size_t)c_tiles * kTile32);
    } else {
        L.n_tiles = (NT + kTile64 - 1) / kTile64;
        L.n_chunks = (N + kTile64 - 1) / kTile64;
        L.n_pts = L.n_tiles * kTile64;
        L.n_src_groups = L.n_chunks;
        L.n_src_pts = L.n_chunks * kTile64;
        int64_t gmax = (int64_t)pl.num_sms * near64_occupancy_ctas();
        if (g_cap > 0 && gmax > g_cap) gmax = g_cap;
        L.Ln = near_partition(L.n_tiles, L.n_chunks, n_img, gmax, ipc);
        const bool layers = pl.lc_tiles > 0;
        const int64_t c_tiles = layers ? pl.lc_tiles : pl.n_check_tiles;
        L.Lc = near_partition(c_tiles, L.n_chunks, layers ? pl.lc_img : n_img, gmax,
                              g_cap > 0 ? 1 : kCheckItemsPerCta);
        // the symmetric float64 kernel: charges, block image set, a normal (growing) scratch
        L.sym = false;
        const int pk = pl.opt.pair_kernel;
        if (!sep && !(pl.Rb > 0.0) && g_cap == 0 && pk != PSUM_PAIRS_ONE_SIDED &&
            (pk == PSUM_PAIRS_SYMMETRIC || L.n_tiles >= kSymMinTiles64)) {
            std::vector<SymSys> one(1);
            one[0].tile0 = 0;
            one[0].n_tiles = L.n_tiles;
            one[0].n_chunks = L.n_chunks;
            one[0].last_n = (int)(N - (L.n_chunks - 1) * kTile64);
            one[0].shift0 = 0;
            one[0].n_img = n_img;
            L.S = sym_partition(one, (int64_t)pl.num_sms * near64s_occupancy_ctas(), kTile64);
            sym_bands(L, kTile64, pl.sym_band_bytes);
            L.sym = true;
        }
        L.ka = L.va = L.kb = L.vb = L.hist = nullptr;
        L.pk32 = L.pk32lo = nullptr;
        L.org = nullptr;
        L.ext = nullptr;
        L.xs = nullptr;
        L.pk64 = b.take<double4_32a>((size_t)L.n_src_pts);
        if (sep) L.tpk64 = b.take<double4_32a>((size_t)L.n_pts);
        L.part_n = b.take<double>(L.sym ? L.S.doubles : (size_t)L.n_tiles * L.Ln.max_contrib * 4 * kTile64);
        L.part_c = b.take<double>((size_t)c_tiles * L.Lc.max_contrib * kTile64);
        L.phi_c = b.take<double>((size_t)c_tiles * kTile64);
    }
    L.phi_n = b.take<double>((size_t)L.n_pts);
    L.grad_n = b.take<double>(3 * (size_t)L.n_pts);
    L.nblk_val = reduce_blocks(N, pl.num_sms);
    L.nblk_mean = mean_blocks(N, pl.num_sms);
    L.val_part = b.take<double>(2 * (size_t)L.nblk_val);
    L.mean_part = b.take<double>((size_t)L.nblk_mean);
    L.f = b.take<double>((size_t)pl.opt.M);
    // the status word and the pair launches' work-item counters
    int* flags = b.take<int>(8);
    L.eval_status = flags;
    L.Ln.counter = flags + 1;
    L.Lc.counter = flags + 2;
    L.Ln.status = L.Lc.status = flags;
    L.Ln.n_status = L.Lc.n_status = 1;
    L.S.counter = flags + 1;
    L.S.status = flags;
    L.S.n_status = 1;
    L.far_phi = L.far_grad = L.w_part = L.w = L.u = L.psi = L.gpsi = L.part_b = nullptr;
    L.chk_src32 = nullptr;
    L.chk_src32lo = nullptr;
    L.chk_src64 = nullptr;
    L.nblk_mom = 0;
    if (backward) {
        // the check points as sources: the two-layer sets (float32 packing with layers) or the 2M points
        const bool bk_layers = fp32 && pl.bk_chunks > 0;
        const int n_img = bk_layers ? pl.bk_lmax : pl.n_images;
        const int64_t n_chk_chunks = bk_layers ? (int64_t)pl.bk_chunks
                                               : fp32 ? (int64_t)pl.n_check_tiles * kTgt32 : (int64_t)pl.n_check_tiles;
        const int64_t gmax = (int64_t)pl.num_sms *
                             (fp32 ? near32_occupancy_ctas(n_img, 0, false, pl.opt.precision == PSUM_FF)
                                   : near64_occupancy_ctas());
        L.Lb = near_partition(L.n_tiles, n_chk_chunks, n_img, gmax);
        L.Lb.tab.one.tau2 = coincident_r2(pl.opt.d);
        L.Lb.counter = flags + 3;
        L.Lb.status = flags;
        L.Lb.n_status = 1;
        L.nblk_mom = moments_blocks(N);
        L.far_phi = b.take<double>((size_t)N);
        L.far_grad = b.take<double>(3 * (size_t)N);
        L.w_part = b.take<double>((size_t)L.nblk_mom * pl.P);
        L.w = b.take<double>((size_t)pl.P);
        L.u = b.take<double>((size_t)pl.opt.M);
        L.psi = b.take<double>((size_t)L.n_pts);
        L.gpsi = b.take<double>(3 * (size_t)L.n_pts);
        const int tile = fp32 ? kTile32 : kTile64;
        L.part_b = b.take<double>((size_t)L.n_tiles * L.Lb.max_contrib * 4 * tile);
        if (fp32) {
            L.chk_src32 = b.take<float4>(2 * (size_t)n_chk_chunks * kNearChunk);
            if (pl.opt.precision == PSUM_FF) L.chk_src32lo = b.take<float4>(2 * (size_t)n_chk_chunks * kNearChunk);
        } else {
            L.chk_src64 = b.take<double4_32a>((size_t)n_chk_chunks * kNearChunk);
        }
    }
    return b.off + 256;
}

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&old_);
        if (old_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != old_) cudaSetDevice(old_);
    }

   private:
    int old_ = 0;
};

#define TRY(expr)                                  \
    do {                                           \
        cudaError_t e_ = (expr);                   \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

int ensure_scratch(Plan& pl, size_t need, int* fail_allocs = nullptr) {
    if (need <= pl.scratch.bytes) return PSUM_OK;
    cudaFree(pl.scratch.ptr);              // synchronises: no queued kernel still uses the old buffer
    pl.scratch.ptr = nullptr;
    pl.scratch.bytes = 0;
    if (fail_allocs && *fail_allocs > 0) {   // test hook: this growth fails as cudaMalloc would
        --*fail_allocs;
        return PSUM_ERR_NOMEM;
    }
    TRY(cudaMalloc(&pl.scratch.ptr, need));
    pl.scratch.bytes = need;
    return PSUM_OK;
}

// Algorithm "get" on the device for the charges (x, q), with the scratch laid out in L;
// every kernel is queued on `st`.
int queue_forward(psum_plan_s* h, int64_t N, const double* x, const double* q, double* phi, double* grad,
                  const Layout& L, cudaStream_t st, int64_t T = -1, const double* y = nullptr) {
    const bool sep = y != nullptr;
    Plan& pl = h->pl;
    const psum_opts& o = pl.opt;
    const bool fp32 = o.precision != PSUM_FP64;       // float32 packing (FP32C and FF)
    const bool ff = o.precision == PSUM_FF;
    const int M = o.M, P = pl.P;
    if (h->profile) TRY(cudaEventRecord(h->ev[0], st));
    // the block's box mean needs only the caller's charges: on the second side stream (least
    // urgent priority) from the start, beside validation, sort and packing; the ball's mean
    // reads the sorted order and forks with the check sums below
    const bool zero_mean = o.mean_mode == PSUM_MEAN_ZERO;
    const bool early_mean = zero_mean && !(pl.Rb > 0.0);
    if (early_mean) {
        cudaStream_t s2 = h->side2;
        TRY(cudaEventRecord(h->fork0, st));
        TRY(cudaStreamWaitEvent(s2, h->fork0, 0));
        const double H[3] = {0.5 * (2 * o.K[0] + 1) * o.d[0], 0.5 * (2 * o.K[1] + 1) * o.d[1],
                             0.5 * (2 * o.K[2] + 1) * o.d[2]};
        TRY(launch_box_mean(x, q, N, H, L.mean_part, L.nblk_mean, s2));
        TRY(cudaEventRecord(h->join2, s2));
        h->launches += 1;
    }
    // the status word must start at zero; every other buffer is written before it is read
    TRY(cudaMemsetAsync(L.eval_status, 0, sizeof(int), st));
    TRY(launch_validate(x, q, N, o.d, L.val_part, L.nblk_val, L.eval_status, st));
    h->launches += 2;
    const int* perm = nullptr;
    if (fp32) {
        TRY(launch_curve_sort(x, N, o.d, L.ka, L.va, L.kb, L.vb, L.hist, st));
        perm = (const int*)L.va;
        TRY(launch_pack32(x, q, L.va, N, L.n_src_groups, L.pk32, L.pk32lo, L.org, st, L.xs, L.ext));
        h->launches += curve_sort_launches(N) + 1;
    } else {
        TRY(launch_pack64(x, q, N, L.n_src_pts, L.pk64, st));
        h->launches += 1;
    }
    // separate evaluation points: validated, sorted and packed like the charges, without charges
    const double* ex = sep ? y : x;              // evaluation points, caller order
    const int* eperm = perm;
    if (sep) {
        TRY(launch_validate_points(y, T, o.d, L.nblk_val, L.eval_status, st));
        h->launches += 1;
        if (fp32) {
            TRY(launch_curve_sort(y, T, o.d, L.tka, L.tva, L.tkb, L.tvb, L.thist, st));
            eperm = (const int*)L.tva;
            TRY(launch_pack32(y, nullptr, L.tva, T, L.n_tiles * kTgt32, L.tpk32, L.tpk32lo, L.torg, st));
            h->launches += curve_sort_launches(T) + 1;
        } else {
            TRY(launch_pack64(y, nullptr, T, L.n_pts, L.tpk64, st));
            h->launches += 1;
        }
    }
    const float4* thi = sep ? L.tpk32 : L.pk32;
    const float4* tlo = sep ? L.tpk32lo : L.pk32lo;
    const double* tor = sep ? L.torg : L.org;
    const double4_32a* t64 = sep ? L.tpk64 : L.pk64;
    if (h->profile) TRY(cudaEventRecord(h->ev[1], st));
    // fork: the side stream (least urgent priority) waits for the packing, then takes the
    // check-point sums, their reduction and the box mean while the charge kernel runs first
    TRY(cudaEventRecord(h->fork, st));
    if (L.sym) {
        // band by band: the pair kernel writes the band's slots, the reduction adds them to the
        // near-field sums in a fixed order (the first band sets them) before the next band
        // reuses the slots; the last band's reduction runs after the kernel's timing event
        for (int64_t k = 0; k < L.sym_bands; ++k) {
            const NearSymLaunch S = sym_band_launch(L, k, h->inject_timeout, h->debug_limit);
            if (fp32)
                TRY(launch_near32s(L.pk32, L.pk32lo, L.org, L.ext, pl.d_shifts, L.part_n, S, st, ff,
                                   refined_terms(pl)));
            else
                TRY(launch_near64s(L.pk64, pl.d_shifts, L.part_n, S, st));
            if (k + 1 < L.sym_bands) TRY(launch_sym_reduce(L.part_n, N, S, L.phi_n, L.grad_n, st, !fp32, k > 0));
        }
        h->launches += 2 * L.sym_bands - 2;   // beyond the one kernel and one reduction counted below
    } else if (fp32) {
        NearPlanLaunch Ln = L.Ln;
        Ln.inject = h->inject_timeout ? 1 : 0;
        Ln.debug_limit = h->debug_limit;
        TRY(launch_near32(true, L.pk32, L.pk32lo, L.org, thi, tlo, tor, pl.d_shifts, L.part_n, Ln, st, 0, L.xs,
                          pl.Rb, ff));
    } else {
        TRY(launch_near64(true, L.pk64, t64, pl.d_shifts, L.part_n, L.Ln, st, pl.Rb));
    }
    if (h->profile) TRY(cudaEventRecord(h->ev[2], st));
    cudaStream_t sd = h->side;
    TRY(cudaStreamWaitEvent(sd, h->fork, 0));
    const bool layers = pl.lc_tiles > 0;
    if (layers && !fp32) {
        TRY(launch_near64(false, L.pk64, (const double4_32a*)pl.d_lc_tgt, pl.d_lc_shifts, L.part_c, L.Lc, sd, 0.0,
                          pl.d_lc_w, kCheckClasses));
    } else if (layers) {
        const float4* ct = (const float4*)pl.d_lc_tgt;
        const size_t half = 2 * (size_t)pl.lc_tiles * kTile32;         // hi parts, then lo parts
        TRY(launch_near32(false, L.pk32, L.pk32lo, L.org, ct, ct + half, pl.d_lc_org, pl.d_lc_shifts, L.part_c,
                          L.Lc, sd, check_variant(pl), nullptr, 0.0, ff, pl.d_lc_gmask, pl.d_lc_w, kCheckClasses,
                          pl.d_lc_sub));
    } else if (fp32) {
        const float4* ct = (const float4*)pl.d_check_tgt;
        const size_t half = 2 * (size_t)pl.n_check_tiles * kTile32;    // hi parts, then lo parts
        TRY(launch_near32(false, L.pk32, L.pk32lo, L.org, ct, ct + half, pl.d_check_org, pl.d_shifts, L.part_c,
                          L.Lc, sd, check_variant(pl), L.xs, pl.Rb, ff));
    } else {
        TRY(launch_near64(false, L.pk64, (const double4_32a*)pl.d_check_tgt, pl.d_shifts, L.part_c, L.Lc, sd,
                          pl.Rb));
    }
    const int tile = fp32 ? kTile32 : kTile64;
    TRY(launch_near_reduce(L.part_c, layers ? (int64_t)pl.lc_tiles * tile : pl.n_check, tile, 1, L.Lc, L.phi_c,
                           nullptr, sd));
    TRY(cudaEventRecord(h->join, sd));
    // the ball's box mean on the second side stream, beside the check sums
    if (zero_mean && !early_mean) {
        cudaStream_t s2 = h->side2;
        TRY(cudaStreamWaitEvent(s2, h->fork, 0));
        TRY(launch_box_mean_ball(x, q, fp32 ? L.va : nullptr, N, o.d, o.K, pl.Rb, L.mean_part, L.nblk_mean, s2));
        TRY(cudaEventRecord(h->join2, s2));
        h->launches += 1;
    }
    if (L.sym)
        TRY(launch_sym_reduce(L.part_n, N, sym_band_launch(L, L.sym_bands - 1, false, h->debug_limit), L.phi_n,
                              L.grad_n, st, !fp32, L.sym_bands > 1));
    else
        TRY(launch_near_reduce(L.part_n, sep ? T : N, tile, 4, L.Ln, L.phi_n, L.grad_n, st));
    h->launches += 4;   // two near-field kernels, two reductions
    // join: the fit needs the check sums and the mean
    TRY(cudaStreamWaitEvent(st, h->join, 0));
    if (zero_mean) TRY(cudaStreamWaitEvent(st, h->join2, 0));
    if (h->profile) TRY(cudaEventRecord(h->ev[3], st));
    TRY(launch_project(pl.d_pinv, P - 1, M, L.phi_c, layers ? pl.d_lc_pos : pl.d_check_pos, L.f, pl.d_C, st,
                       layers));
    TRY(launch_constant(pl.d_C, pl.d_Rbox, P, L.mean_part, L.nblk_mean, 1.0 / (o.d[0] * o.d[1] * o.d[2]),
                        zero_mean ? 1 : 0, st));
    if (h->profile) TRY(cudaEventRecord(h->ev[4], st));
    const int64_t NE = sep ? T : N;
    if (o.basis == PSUM_BASIS_RBF)
        TRY(launch_far_rbf(ex, NE, eperm, L.phi_n, grad ? L.grad_n : nullptr, pl.d_C, pl.d_rbf, pl.P - 1,
                           L.eval_status, phi, grad, L.eval_status, st));
    else
        TRY(launch_far_combine(ex, NE, eperm, L.phi_n, grad ? L.grad_n : nullptr, pl.d_C, o.p, 1.0 / pl.R0,
                               pl.d_shtab64, o.precision == PSUM_FP32C ? pl.d_shtab32 : nullptr, L.eval_status,
                               phi, grad, L.eval_status, st));
    k_status_merge<<<1, 1, 0, st>>>(L.eval_status, pl.d_status);
    TRY(cudaGetLastError());
    h->launches += 5;   // right-hand side, projection, constant, far field, status merge
    if (h->profile) TRY(cudaEventRecord(h->ev[5], st));
    return PSUM_OK;
}

int eval_device(psum_plan_s* h, int64_t N, const double* x, const double* q, double* phi, double* grad,
                cudaStream_t st) {
    Plan& pl = h->pl;
    Layout L;
    int rs = ensure_scratch(pl, layout(pl, N, nullptr, L), &h->fail_allocs);
    if (rs != PSUM_OK) return rs;
    layout(pl, N, (char*)pl.scratch.ptr, L);
    return queue_forward(h, N, x, q, phi, grad, L, st);
}

int eval_points_device(psum_plan_s* h, int64_t N, const double* x, const double* q, int64_t T, const double* y,
                       double* phi, double* grad, cudaStream_t st) {
    Plan& pl = h->pl;
    Layout L;
    int rs = ensure_scratch(pl, layout(pl, N, nullptr, L, false, 0, T), &h->fail_allocs);
    if (rs != PSUM_OK) return rs;
    layout(pl, N, (char*)pl.scratch.ptr, L, false, 0, T);
    return queue_forward(h, N, x, q, phi, grad, L, st, T, y);
}

// The energy derivatives (the exact adjoint of the discrete method: moments w = sum q R^(x/R0),
// u = (A^+)^T w, psi from the check points carrying -u and u) with the far-field coefficients C
// of the evaluation that produced phi and grad.
int backward_device(psum_plan_s* h, int64_t N, const double* x, const double* q, const double* phi,
                    const double* grad, const double* C, const double* gE, double* dEdq, double* dEdx,
                    cudaStream_t st) {
    Plan& pl = h->pl;
    const psum_opts& o = pl.opt;
    Layout L;
    int rs = ensure_scratch(pl, layout(pl, N, nullptr, L, true), &h->fail_allocs);
    if (rs != PSUM_OK) return rs;
    layout(pl, N, (char*)pl.scratch.ptr, L, true);
    const bool fp32 = o.precision != PSUM_FP64;       // float32 packing (FP32C and FF)
    const bool ff = o.precision == PSUM_FF;
    const int M = o.M, P = pl.P;
    if (moments_smem(o.p) > 48 * 1024) TRY(set_moments_smem(moments_smem(o.p)));
    TRY(cudaMemsetAsync(L.eval_status, 0, sizeof(int), st));
    const int* perm = nullptr;
    if (fp32) {
        TRY(launch_curve_sort(x, N, o.d, L.ka, L.va, L.kb, L.vb, L.hist, st));
        perm = (const int*)L.va;
        TRY(launch_pack32(x, q, L.va, N, L.n_src_groups, L.pk32, L.pk32lo, L.org, st));
        h->launches += curve_sort_launches(N) + 1;
    } else {
        TRY(launch_pack64(x, q, N, L.n_src_pts, L.pk64, st));
        h->launches += 1;
    }
    // moments w and the far field at the charges; u = (A^+)^T w
    TRY(launch_moments(x, q, N, C, o.p, 1.0 / pl.R0, pl.d_shtab64, L.far_phi, L.far_grad, L.w_part,
                       L.nblk_mom, L.w, st));
    TRY(launch_adjoint(pl.d_pinv, P - 1, M, L.w, L.u, st));
    h->launches += 3;
    // psi and grad psi at the charges: the check points as sources
    const int tile = fp32 ? kTile32 : kTile64;
    if (fp32 && pl.bk_chunks > 0) {
        // two-layer check sources: each chunk with its (class, side) image list
        const size_t n_bk = (size_t)pl.bk_chunks * kNearChunk;
        const float4* bk = (const float4*)pl.d_bk_pk;
        TRY(launch_check_sources32(bk, bk + 2 * n_bk, pl.d_bk_slot, (int64_t)n_bk, M, L.u, L.chk_src32, L.chk_src32lo,
                                   st, true));
        TRY(launch_near32(true, L.chk_src32, ff ? L.chk_src32lo : bk + 2 * n_bk, pl.d_bk_org, L.pk32, L.pk32lo, L.org,
                          pl.d_bk_shifts, L.part_b, L.Lb, st, 0, nullptr, 0.0, ff, nullptr, nullptr, 1, nullptr,
                          pl.d_bk_img0, pl.d_bk_nimg));
    } else if (fp32) {
        const size_t n_chk_pts = (size_t)pl.n_check_tiles * kTile32;
        const float4* chk = (const float4*)pl.d_check_tgt;
        TRY(launch_check_sources32(chk, chk + 2 * n_chk_pts, pl.d_check_inv, (int64_t)n_chk_pts, M, L.u,
                                   L.chk_src32, L.chk_src32lo, st));
        TRY(launch_near32(true, L.chk_src32, ff ? L.chk_src32lo : chk + 2 * n_chk_pts, pl.d_check_org, L.pk32,
                          L.pk32lo, L.org, pl.d_shifts, L.part_b, L.Lb, st, 0, nullptr, 0.0, ff));
    } else {
        const size_t n_chk_pts = (size_t)pl.n_check_tiles * kTile64;
        TRY(launch_check_sources64((const double4_32a*)pl.d_check_tgt, (int64_t)n_chk_pts, M, L.u, L.chk_src64, st));
        TRY(launch_near64(true, L.chk_src64, L.pk64, pl.d_shifts, L.part_b, L.Lb, st));
    }
    TRY(launch_near_reduce(L.part_b, N, tile, 4, L.Lb, L.psi, L.gpsi, st));
    TRY(launch_backward_combine(N, perm, q, phi, grad, L.far_phi, L.far_grad, L.psi, L.gpsi, gE, dEdq, dEdx, st));
    k_status_merge<<<1, 1, 0, st>>>(L.eval_status, pl.d_status);
    TRY(cudaGetLastError());
    h->launches += 5;
    return PSUM_OK;
}

bool valid_opts(const psum_opts* o) {
    if (!o) return false;
    for (int k = 0; k < 3; ++k) {
        if (!(o->d[k] > 0.0) || !std::isfinite(o->d[k])) return false;
        if (o->K[k] < 0 || o->K[k] > 3) return false;
    }
    if (o->p < 1 || o->p > kMaxDegree) return false;
    const int P = (o->p + 1) * (o->p + 1);
    if (o->points != PSUM_POINTS_FIBONACCI && o->points != PSUM_POINTS_GAUSS) return false;
    if (o->points == PSUM_POINTS_GAUSS) {
        if (o->M != 0 && o->M != (o->p + 1) * (2 * o->p + 1)) return false;
    } else if (o->M < P - 1 || o->M > 100000) {
        return false;
    }
    if (!(o->lambda == 0.0 || (o->lambda > 1.0 && o->lambda <= 8.0))) return false;
    if (o->basis != PSUM_BASIS_SPHERICAL && o->basis != PSUM_BASIS_RBF) return false;
    if (o->basis == PSUM_BASIS_RBF) {
        const int S = o->n_rbf == 0 ? 256 : o->n_rbf;
        const int Mv = o->points == PSUM_POINTS_GAUSS ? (o->p + 1) * (2 * o->p + 1) : o->M;
        if (S < 1 || S > 4096 || Mv < S) return false;
        if (!(o->rbf_radius == 0.0 || (o->rbf_radius > 1.0 && o->rbf_radius <= 100.0))) return false;
    }
    if (o->lambda > 0.0) {
        // the covering block must stay within the image table
        const double R0 = 0.5 * std::sqrt(o->d[0] * o->d[0] + o->d[1] * o->d[1] + o->d[2] * o->d[2]);
        int64_t n = 1;
        for (int k = 0; k < 3; ++k) n *= 2 * (int64_t)std::ceil(o->lambda * R0 / o->d[k] + 0.5) + 1;
        if (n > 100000) return false;
    }
    if (o->precision != PSUM_FP64 && o->precision != PSUM_FP32C && o->precision != PSUM_FF) return false;
    if (o->pair_kernel != PSUM_PAIRS_AUTO && o->pair_kernel != PSUM_PAIRS_ONE_SIDED &&
        o->pair_kernel != PSUM_PAIRS_SYMMETRIC)
        return false;
    if (o->check_form != PSUM_CHECKS_AUTO && o->check_form != PSUM_CHECKS_POINTS &&
        o->check_form != PSUM_CHECKS_LAYERS)
        return false;
    if (o->check_form == PSUM_CHECKS_LAYERS && o->lambda > 0.0) return false;
    if (o->fp32_terms != PSUM_TERMS_FAST && o->fp32_terms != PSUM_TERMS_REFINED) return false;
    if (o->mean_mode != PSUM_MEAN_ZERO && o->mean_mode != PSUM_MEAN_NONE) return false;
    return true;
}

}  // namespace

extern "C" {

void psum_opts_default(psum_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->d[0] = o->d[1] = o->d[2] = 1.0;
    o->p = 8;
    o->M = 200;
    o->precision = PSUM_FP64;
    o->mean_mode = PSUM_MEAN_ZERO;
    o->K[0] = o->K[1] = o->K[2] = 1;
    o->points = PSUM_POINTS_FIBONACCI;
    o->lambda = 0.0;
    o->basis = PSUM_BASIS_SPHERICAL;
    o->n_rbf = 256;
    o->rbf_radius = 0.0;
    o->pair_kernel = PSUM_PAIRS_AUTO;
    o->check_form = PSUM_CHECKS_AUTO;
    o->fp32_terms = PSUM_TERMS_FAST;
}

}  // extern "C"

namespace {

// Plan creation; `stored` (may be null) carries a factorisation read by psum_plan_load.
int create_plan(const psum_opts* o, psum_plan_t* out, const Plan* stored) {
    if (!out || !valid_opts(o)) return PSUM_ERR_ARG;
    psum_opts oo = *o;
    if (oo.points == PSUM_POINTS_GAUSS) oo.M = (oo.p + 1) * (2 * oo.p + 1);
    if (oo.basis == PSUM_BASIS_RBF && oo.n_rbf == 0) oo.n_rbf = 256;
    psum_plan_s* h = new (std::nothrow) psum_plan_s();
    if (!h) return PSUM_ERR_NOMEM;
    if (stored) {
        h->pl.preset_pinv = stored->preset_pinv;
        h->pl.preset_rank = stored->preset_rank;
        h->pl.preset_cond = stored->preset_cond;
        h->pl.preset_geom = stored->preset_geom;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        delete h;
        return PSUM_ERR_CUDA;
    }
    h->pl.device = dev;
    cudaDeviceGetAttribute(&h->pl.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (h->pl.num_sms < 1) h->pl.num_sms = 1;
    const int st = build_plan(oo, h->pl);
    if (st != PSUM_OK) {
        free_plan_device(h->pl);
        delete h;
        return st;
    }
    h->pl.preset_pinv.clear();
    h->pl.preset_pinv.shrink_to_fit();
    for (auto& e : h->ev) cudaEventCreate(&e);
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);   // lo: the least urgent priority
    if (cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->side2, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join2, cudaEventDisableTiming) != cudaSuccess) {
        psum_destroy(h);
        return PSUM_ERR_CUDA;
    }
    *out = h;
    return PSUM_OK;
}

// Plan files: a magic word, the size of psum_opts, the plan's options, the fingerprint of its
// check points, the rank and condition estimate, the (P-1) x M pseudo-inverse, and an FNV-1a
// checksum of all that.  Little-endian IEEE doubles as the host writes them.
constexpr char kPlanMagic[8] = {'P', 'S', 'U', 'M', 'P', 'L', 'N', '1'};

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

extern "C" {

int psum_plan_create_ex(const psum_opts* o, psum_plan_t* out) { return create_plan(o, out, nullptr); }

int psum_plan_save(psum_plan_t h, const char* path) {
    if (!h || !path) return PSUM_ERR_ARG;
    const Plan& pl = h->pl;
    std::vector<unsigned char> buf;
    auto put = [&buf](const void* p, size_t n) {
        const unsigned char* c = (const unsigned char*)p;
        buf.insert(buf.end(), c, c + n);
    };
    const uint32_t ob = (uint32_t)sizeof(psum_opts);
    const int32_t rank = pl.rank;
    const uint64_t npinv = pl.pinv.size();
    put(kPlanMagic, sizeof kPlanMagic);
    put(&ob, sizeof ob);
    put(&pl.opt, sizeof pl.opt);
    put(&pl.geom_hash, sizeof pl.geom_hash);
    put(&rank, sizeof rank);
    put(&pl.cond_est, sizeof pl.cond_est);
    put(&npinv, sizeof npinv);
    put(pl.pinv.data(), sizeof(double) * npinv);
    const uint64_t sum = fnv1a(buf.data(), buf.size());
    put(&sum, sizeof sum);
    FILE* f = std::fopen(path, "wb");
    if (!f) return PSUM_ERR_IO;
    const size_t wrote = std::fwrite(buf.data(), 1, buf.size(), f);
    const int closed = std::fclose(f);
    return wrote == buf.size() && closed == 0 ? PSUM_OK : PSUM_ERR_IO;
}

int psum_plan_load(const char* path, psum_plan_t* out) {
    if (!path || !out) return PSUM_ERR_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return PSUM_ERR_IO;
    std::vector<unsigned char> buf;
    unsigned char chunk[1 << 16];
    size_t n;
    while ((n = std::fread(chunk, 1, sizeof chunk, f)) > 0) buf.insert(buf.end(), chunk, chunk + n);
    std::fclose(f);
    size_t off = 0;
    auto get = [&](void* p, size_t k) {
        if (off + k > buf.size()) return false;
        std::memcpy(p, buf.data() + off, k);
        off += k;
        return true;
    };
    char magic[8];
    uint32_t ob = 0;
    psum_opts o;
    Plan stored;
    int32_t rank = 0;
    uint64_t npinv = 0, sum = 0;
    if (!get(magic, sizeof magic) || std::memcmp(magic, kPlanMagic, sizeof magic) != 0) return PSUM_ERR_IO;
    if (!get(&ob, sizeof ob) || ob != sizeof(psum_opts) || !get(&o, sizeof o)) return PSUM_ERR_IO;
    if (!get(&stored.preset_geom, sizeof stored.preset_geom) || !get(&rank, sizeof rank) ||
        !get(&stored.preset_cond, sizeof stored.preset_cond) || !get(&npinv, sizeof npinv))
        return PSUM_ERR_IO;
    if (npinv == 0 || npinv > (uint64_t)1 << 32 || off + sizeof(double) * npinv + sizeof sum != buf.size())
        return PSUM_ERR_IO;
    stored.preset_pinv.resize(npinv);
    get(stored.preset_pinv.data(), sizeof(double) * npinv);
    const uint64_t expect = fnv1a(buf.data(), off);
    if (!get(&sum, sizeof sum) || sum != expect) return PSUM_ERR_IO;
    if (!valid_opts(&o)) return PSUM_ERR_IO;
    stored.preset_rank = rank;
    return create_plan(&o, out, &stored);
}

int psum_plan_create(double d1, double d2, double d3, int p, int M, psum_plan_t* out) {
    psum_opts o;
    psum_opts_default(&o);
    o.d[0] = d1;
    o.d[1] = d2;
    o.d[2] = d3;
    o.p = p;
    o.M = M;
    return psum_plan_create_ex(&o, out);
}

int psum_eval(psum_plan_t h, int64_t N, const double* x, const double* q, double* phi, double* grad,
              void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || !x || !q || !phi) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    return eval_device(h, N, x, q, phi, grad, (cudaStream_t)stream);
}

int psum_eval_graph(psum_plan_t h, int64_t N, const double* x, const double* q, double* phi, double* grad,
                    void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || !x || !q || !phi) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    Plan& pl = h->pl;
    cudaStream_t st = (cudaStream_t)stream;
    Layout L;
    int rs = ensure_scratch(pl, layout(pl, N, nullptr, L), &h->fail_allocs);     // outside any capture
    if (rs != PSUM_OK) return rs;
    const void* key[6] = {x, q, phi, grad, pl.scratch.ptr, (const void*)(intptr_t)h->inject_timeout};
    bool same = h->gexec != nullptr && h->gN == N;
    for (int k = 0; k < 6 && same; ++k) same = h->gkey[k] == key[k];
    if (!same) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        if (!h->cap) TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
        layout(pl, N, (char*)pl.scratch.ptr, L);
        const bool prof = h->profile;
        h->profile = false;                       // no timing events inside the graph
        const int64_t before = h->launches;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            h->profile = prof;
            return cuda_status(e);
        }
        const int s = queue_forward(h, N, x, q, phi, grad, L, h->cap);
        e = cudaStreamEndCapture(h->cap, &graph);
        h->profile = prof;
        h->glaunches = h->launches - before;
        h->launches = before;                     // capturing queues nothing on the device
        if (s != PSUM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        TRY(e);
        e = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
        TRY(e);
        for (int k = 0; k < 6; ++k) h->gkey[k] = key[k];
        h->gN = N;
    }
    TRY(cudaGraphLaunch(h->gexec, st));
    h->launches += h->glaunches;
    return PSUM_OK;
}

int psum_eval_points(psum_plan_t h, int64_t N, const double* x, const double* q, int64_t T, const double* y,
                     double* phi, double* grad, void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || T < 1 || T > (int64_t)1 << 30 || !x || !q || !y || !phi)
        return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    return eval_points_device(h, N, x, q, T, y, phi, grad, (cudaStream_t)stream);
}

int psum_sync(psum_plan_t h, void* stream) {
    if (!h) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    cudaStream_t st = (cudaStream_t)stream;
    TRY(cudaMemcpyAsync(h->pl.h_status, h->pl.d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaMemsetAsync(h->pl.d_status, 0, sizeof(int), st));
    TRY(cudaStreamSynchronize(st));
    return map_device_status(*h->pl.h_status);
}

int psum_eval_host(psum_plan_t h, int64_t N, const double* x, const double* q, double* phi, double* grad,
                   void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || !x || !q || !phi) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    Plan& pl = h->pl;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bx = sizeof(double) * 3 * (size_t)N, bq = sizeof(double) * (size_t)N;
    const size_t need = 2 * bx + 2 * bq + 4 * 256;
    if (need > pl.dstage.bytes) {
        cudaFree(pl.dstage.ptr);
        pl.dstage.ptr = nullptr;
        pl.dstage.bytes = 0;
        TRY(cudaMalloc(&pl.dstage.ptr, need));
        pl.dstage.bytes = need;
    }
    Bump b{(char*)pl.dstage.ptr, 0, need};
    double* dx = b.take<double>(3 * (size_t)N);
    double* dq = b.take<double>((size_t)N);
    double* dphi = b.take<double>((size_t)N);
    double* dgrad = b.take<double>(3 * (size_t)N);
    TRY(cudaMemcpyAsync(dx, x, bx, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(dq, q, bq, cudaMemcpyHostToDevice, st));
    int s = eval_device(h, N, dx, dq, dphi, grad ? dgrad : nullptr, st);
    if (s != PSUM_OK) return s;
    TRY(cudaMemcpyAsync(phi, dphi, bq, cudaMemcpyDeviceToHost, st));
    if (grad) TRY(cudaMemcpyAsync(grad, dgrad, bx, cudaMemcpyDeviceToHost, st));
    return psum_sync(h, stream);
}

int psum_energy(psum_plan_t h, int64_t N, const double* q, const double* phi, double* E, void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || !q || !phi || !E) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    Layout L;
    int rs = ensure_scratch(h->pl, layout(h->pl, N, nullptr, L), &h->fail_allocs);
    if (rs != PSUM_OK) return rs;
    layout(h->pl, N, (char*)h->pl.scratch.ptr, L);
    TRY(launch_energy(q, phi, N, L.val_part, L.nblk_val, E, (cudaStream_t)stream));
    h->launches += 2;
    return PSUM_OK;
}

int psum_energy_backward(psum_plan_t h, int64_t N, const double* x, const double* q, const double* phi,
                         const double* grad, const double* gE, double* dEdq, double* dEdx, void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || !x || !q || !phi || !grad || (!dEdq && !dEdx)) return PSUM_ERR_ARG;
    if (h->pl.Rb > 0.0) return PSUM_ERR_ARG;   // the adjoint assumes the untrimmed near block
    if (h->pl.opt.basis != PSUM_BASIS_SPHERICAL) return PSUM_ERR_ARG;   // and the solid-harmonic moments
    DeviceGuard g(h->pl.device);
    return backward_device(h, N, x, q, phi, grad, h->pl.d_C, gE, dEdq, dEdx, (cudaStream_t)stream);
}

int psum_coeffs_device(psum_plan_t h, double* C, void* stream) {
    if (!h || !C) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    TRY(cudaMemcpyAsync(C, h->pl.d_C, sizeof(double) * h->pl.P, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PSUM_OK;
}

int psum_energy_backward_c(psum_plan_t h, int64_t N, const double* x, const double* q, const double* phi,
                           const double* grad, const double* C, const double* gE, double* dEdq, double* dEdx,
                           void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || !x || !q || !phi || !grad || !C || (!dEdq && !dEdx))
        return PSUM_ERR_ARG;
    if (h->pl.Rb > 0.0) return PSUM_ERR_ARG;
    if (h->pl.opt.basis != PSUM_BASIS_SPHERICAL) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    return backward_device(h, N, x, q, phi, grad, C, gE, dEdq, dEdx, (cudaStream_t)stream);
}

int psum_get_coeffs(psum_plan_t h, double* C, void* stream) {
    if (!h || !C) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    cudaStream_t st = (cudaStream_t)stream;
    TRY(cudaMemcpyAsync(C, h->pl.d_C, sizeof(double) * h->pl.P, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    return PSUM_OK;
}

int psum_plan_info(psum_plan_t h, psum_info* info) {
    if (!h || !info) return PSUM_ERR_ARG;
    const Plan& pl = h->pl;
    std::memset(info, 0, sizeof(*info));
    for (int k = 0; k < 3; ++k) {
        info->d[k] = pl.opt.d[k];
        info->K[k] = pl.opt.K[k];
    }
    info->R0 = pl.R0;
    info->lambda_eff = pl.lambda_eff;
    info->cond_est = pl.cond_est;
    info->rank = pl.rank;
    info->p = pl.opt.p;
    info->P = pl.P;
    info->M = pl.opt.M;
    info->n_images = pl.n_images;
    info->precision = pl.opt.precision;
    info->mean_mode = pl.opt.mean_mode;
    return PSUM_OK;
}

int psum_pair_kernel(psum_plan_t h, int64_t N, int* kernel, int* image_groups) {
    if (!h || !kernel || N < 0) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    Layout L{};
    layout(h->pl, N, nullptr, L);
    *kernel = L.sym ? PSUM_PAIRS_SYMMETRIC : PSUM_PAIRS_ONE_SIDED;
    if (image_groups) *image_groups = L.sym ? L.S.tab.one.n_g : 0;
    return PSUM_OK;
}

int psum_scratch_bytes(psum_plan_t h, int64_t N, int64_t* bytes, int* bands) {
    if (!h || !bytes || N < 1) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    Layout L{};
    *bytes = (int64_t)layout(h->pl, N, nullptr, L);
    if (bands) *bands = L.sym ? (int)L.sym_bands : 0;
    return PSUM_OK;
}

int psum_debug_bounds_limit(psum_plan_t h, int64_t doubles) {
    if (!h || doubles < 0) return PSUM_ERR_ARG;
    h->debug_limit = doubles;
    return PSUM_OK;
}

int psum_debug_checks(void) { return PSUM_DEBUG_CHECKS; }

int psum_debug_fail_allocs(psum_plan_t h, int count) {
    if (!h || count < 0) return PSUM_ERR_ARG;
    h->fail_allocs = count;
    return PSUM_OK;
}

int psum_debug_band_bytes(psum_plan_t h, int64_t bytes) {
    if (!h || bytes < 0) return PSUM_ERR_ARG;
    h->pl.sym_band_bytes = (size_t)bytes;
    return PSUM_OK;
}

int psum_check_form(psum_plan_t h, int* form) {
    if (!h || !form) return PSUM_ERR_ARG;
    *form = h->pl.lc_tiles > 0 ? PSUM_CHECKS_LAYERS : PSUM_CHECKS_POINTS;
    return PSUM_OK;
}

int psum_debug_inject_timeout(psum_plan_t h, int enable) {
    if (!h) return PSUM_ERR_ARG;
    h->inject_timeout = enable != 0;
    return PSUM_OK;
}

int psum_profile(psum_plan_t h, int enable) {
    if (!h) return PSUM_ERR_ARG;
    h->profile = enable != 0;
    return PSUM_OK;
}

int psum_last_timings(psum_plan_t h, double* ms, void* stream) {
    if (!h || !ms) return PSUM_ERR_ARG;
    if (!h->profile) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    TRY(cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; i < PSUM_NUM_STAGES; ++i) {
        float t = 0.f;
        TRY(cudaEventElapsedTime(&t, h->ev[i], h->ev[i + 1]));
        ms[i] = t;
    }
    return PSUM_OK;
}

int psum_launch_count(psum_plan_t h, int64_t* count) {
    if (!h || !count) return PSUM_ERR_ARG;
    *count = h->launches;
    return PSUM_OK;
}

void psum_destroy(psum_plan_t h) {
    if (!h) return;
    {
        DeviceGuard g(h->pl.device);
        cudaDeviceSynchronize();
        for (auto& e : h->ev)
            if (e) cudaEventDestroy(e);
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        if (h->cap) cudaStreamDestroy(h->cap);
        if (h->side) cudaStreamDestroy(h->side);
        if (h->side2) cudaStreamDestroy(h->side2);
        if (h->fork0) cudaEventDestroy(h->fork0);
        if (h->fork) cudaEventDestroy(h->fork);
        if (h->join) cudaEventDestroy(h->join);
        if (h->join2) cudaEventDestroy(h->join2);
        free_plan_device(h->pl);
    }
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free evaluation (psum_eval_noalloc).
//
// Some callers cannot call cudaMalloc at evaluation time: code that runs inside a
// CUDA stream capture (a graph is being recorded and an allocation would break
// it), real-time loops that cannot afford the device-wide synchronisation a
// cudaMalloc/cudaFree implies, and runtimes that hand out all device memory from
// their own pool.  psum_eval grows its scratch with cudaMalloc the first time a size
// is seen; this variant instead takes all scratch from one file-scope device array
// of kNoAllocBytes, which every GPU that loads the library holds until exit.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = (size_t)16 << 20;     // 16 MiB
constexpr int64_t kNoAllocMaxCtas = 256;                // CTAs (one work item each): bounds the partial sums
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};          // device address of the array, per device

// Once per device, with that device current: the array's name is only a host-side
// stand-in, so its device address must be looked up before a kernel may use it.
int noalloc_scratch(int dev, char** out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return PSUM_ERR_ARG;
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return PSUM_ERR_CUDA;
        g_noalloc_addr[dev] = ptr;
    }
    *out = (char*)g_noalloc_addr[dev];
    return PSUM_OK;
}

int eval_noalloc_device(psum_plan_s* h, int64_t N, const double* x, const double* q, double* phi, double* grad,
                        cudaStream_t st) {
    Plan& pl = h->pl;
    char* base = nullptr;
    int rs = noalloc_scratch(pl.device, &base);
    if (rs != PSUM_OK) return rs;
    Layout L;
    if (layout(pl, N, nullptr, L, false, kNoAllocMaxCtas) > kNoAllocBytes) return PSUM_ERR_ARG;
    layout(pl, N, base, L, false, kNoAllocMaxCtas);
    // the array keeps the previous call's contents; the pipeline zeroes the status word
    // first and writes every other buffer before reading it
    return queue_forward(h, N, x, q, phi, grad, L, st);
}

}  // namespace

extern "C" int psum_eval_noalloc(psum_plan_t h, int64_t N, const double* x, const double* q, double* phi,
                                 double* grad, void* stream) {
    if (!h || N < 1 || N > (int64_t)1 << 30 || !x || !q || !phi) return PSUM_ERR_ARG;
    DeviceGuard g(h->pl.device);
    return eval_noalloc_device(h, N, x, q, phi, grad, (cudaStream_t)stream);
}

extern "C" {

const char* psum_strerror(int s) {
    switch (s) {
        case PSUM_OK: return "ok";
        case PSUM_ERR_ARG: return "invalid argument";
        case PSUM_ERR_NONNEUTRAL: return "charges do not sum to zero (|sum q| > 1e-12 sum |q|)";
        case PSUM_ERR_OUT_OF_BOX: return "a position lies outside the box [-d/2, d/2) or is not finite";
        case PSUM_ERR_RANK: return "the fitting matrix is rank deficient (more check points needed)";
        case PSUM_ERR_CUDA: return "CUDA runtime error";
        case PSUM_ERR_TIMEOUT: return "a device-side wait timed out";
        case PSUM_ERR_NOMEM: return "out of memory";
        case PSUM_ERR_NONFINITE: return "a result or charge is not finite";
        case PSUM_ERR_INTERNAL: return "an internal bounds check refused an access (debug build)";
        case PSUM_ERR_IO: return "a plan file cannot be read or written, or does not match this library";
        default: return "unknown status";
    }
}

}  // extern "C"
