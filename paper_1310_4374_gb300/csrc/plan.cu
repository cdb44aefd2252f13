// Algorithm "set" (Sec. 2.3.1) on the host in float64, and the upload of its
// results to the device.
//
//   step 1: circumradius R0 = |d|/2
//   step 2: M check points on the sphere of radius R0 (spherical Fibonacci lattice)
//   step 3: periodic partners y~_l (one coordinate shifted by one period into S0)
//   step 4: A_lt = R_t(y_l/R0) - R_t(y~_l/R0), t = 2..P (the constant column is
//           identically zero and is dropped, Sec. 3)
//   step 5: column-pivoted Householder QR of A and the pseudo-inverse
//           A^+ = Pi R^-1 Q^T (Eq. 10), so that "get" needs one matrix-vector product
//   step 6: box integrals R_t^(0) by tensor Gauss-Legendre quadrature with
//           floor(p/2)+1 nodes per axis, exact for degree <= p (App. B, Eqs. A1-A2)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "launch.cuh"
#include "mean.cuh"

namespace psum {

static void fibonacci_sphere(int M, double R0, std::vector<double>& Y) {
    Y.resize(3 * (size_t)M);
    const double golden = M_PI * (3.0 - std::sqrt(5.0));
    for (int l = 0; l < M; ++l) {
        const double z = 1.0 - (2.0 * l + 1.0) / M;
        const double rho = std::sqrt(std::max(0.0, 1.0 - z * z));
        const double az = l * golden;
        Y[3 * l + 0] = R0 * rho * std::cos(az);
        Y[3 * l + 1] = R0 * rho * std::sin(az);
        Y[3 * l + 2] = R0 * z;
    }
}

// Partner: shift the coordinate with the largest |y_k|/d_k (first on ties) by one
// period towards the box.
static void partners(const std::vector<double>& Y, const double d[3], std::vector<double>& Yt) {
    const size_t M = Y.size() / 3;
    Yt = Y;
    for (size_t l = 0; l < M; ++l) {
        int k = 0;
        double best = std::fabs(Y[3 * l]) / d[0];
        for (int c = 1; c < 3; ++c) {
            const double v = std::fabs(Y[3 * l + c]) / d[c];
            if (v > best) { best = v; k = c; }
        }
        const double y = Y[3 * l + k];
        Yt[3 * l + k] = y - (y > 0 ? d[k] : (y < 0 ? -d[k] : 0.0));
    }
}

static void basis_values(double x, double y, double z, int p, double* out) {
    sh_visit<false>(x, y, z, p, [&](int n, int m, double v, double, double, double) { out[sh_index(n, m)] = v; });
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w) {
    t.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        // recompute the derivative at the converged node
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = x; p0 = 1.0; }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        t[i] = x;
        w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

// Householder QR with column pivoting of the M x n matrix A (column-major),
// then pinv = Pi R^-1 Q1^T (n x M, row-major).  Returns PSUM_ERR_RANK if
// |R_kk| < 1e-13 |R_11| for some k.
static int qr_pseudo_inverse(std::vector<double>& A, int M, int n, std::vector<double>& pinv, int& rank,
                             double& cond_est) {
    std::vector<int> piv(n);
    std::iota(piv.begin(), piv.end(), 0);
    std::vector<double> beta(n, 0.0), rdiag(n, 0.0);
    auto col = [&](int j) { return A.data() + (size_t)j * M; };
    for (int k = 0; k < n; ++k) {
        // pivot: the remaining column of largest norm (recomputed exactly)
        int jb = k;
        double nb = -1.0;
        for (int j = k; j < n; ++j) {
            const double* c = col(j);
            double s = 0.0;
            for (int i = k; i < M; ++i) s += c[i] * c[i];
            if (s > nb) { nb = s; jb = j; }
        }
        if (jb != k) {
            std::swap_ranges(col(k), col(k) + M, col(jb));
            std::swap(piv[k], piv[jb]);
        }
        double* v = col(k);
        const double norm = std::sqrt(nb);
        const double alpha = v[k] > 0 ? -norm : norm;
        rdiag[k] = alpha;
        if (norm == 0.0) { beta[k] = 0.0; continue; }
        v[k] -= alpha;                          // v = x - alpha e1 (stored in place below the diagonal)
        double vv = 0.0;
        for (int i = k; i < M; ++i) vv += v[i] * v[i];
        beta[k] = vv > 0 ? 2.0 / vv : 0.0;
        for (int j = k + 1; j < n; ++j) {
            double* c = col(j);
            double s = 0.0;
            for (int i = k; i < M; ++i) s += v[i] * c[i];
            s *= beta[k];
            for (int i = k; i < M; ++i) c[i] -= s * v[i];
        }
    }
    const double r11 = std::fabs(rdiag[0]);
    rank = 0;
    double rmin = r11;
    for (int k = 0; k < n; ++k) {
        const double a = std::fabs(rdiag[k]);
        if (!(a >= 1e-13 * r11) || r11 == 0.0) break;
        rank = k + 1;
        rmin = std::min(rmin, a);
    }
    cond_est = rmin > 0 ? r11 / rmin : INFINITY;
    if (rank < n) return PSUM_ERR_RANK;
    // Q1 (M x n): apply H_0 .. H_{n-1} to [I_n; 0] in reverse order
    std::vector<double> Q((size_t)M * n, 0.0);      // column-major
    for (int j = 0; j < n; ++j) Q[(size_t)j * M + j] = 1.0;
    for (int k = n - 1; k >= 0; --k) {
        const double* v = col(k);
        for (int j = 0; j < n; ++j) {
            double* c = Q.data() + (size_t)j * M;
            double s = 0.0;
            for (int i = k; i < M; ++i) s += v[i] * c[i];
            s *= beta[k];
            for (int i = k; i < M; ++i) c[i] -= s * v[i];
        }
    }
    // Z = R^-1 Q1^T by back substitution, R upper-triangular: R_kk = rdiag[k],
    // R_kj (j > k) = A[k][j] after the factorisation.
    pinv.assign((size_t)n * M, 0.0);
    std::vector<double> z(n);
    for (int l = 0; l < M; ++l) {
        for (int k = n - 1; k >= 0; --k) {
            double s = Q[(size_t)k * M + l];
            for (int j = k + 1; j < n; ++j) s -= A[(size_t)j * M + k] * z[j];
            z[k] = s / rdiag[k];
        }
        for (int k = 0; k < n; ++k) pinv[(size_t)piv[k] * M + l] = z[k];
    }
    return PSUM_OK;
}

// Morton order of points inside [-R, R]^3 (host), used to group the check targets.
static uint64_t morton_host(const double* p, double R) {
    uint64_t key = 0;
    uint32_t c[3];
    for (int k = 0; k < 3; ++k) {
        double u = (p[k] / (2.0 * R) + 0.5) * 1024.0;
        int v = (int)std::floor(u);
        c[k] = (uint32_t)std::min(1023, std::max(0, v));
    }
    for (int b = 9; b >= 0; --b)
        for (int k = 0; k < 3; ++k) key = (key << 1) | ((c[k] >> b) & 1u);
    return key;
}

#define PSUM_CUDA_TRY(call)                            \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ == cudaErrorMemoryAllocation) return PSUM_ERR_NOMEM; \
        if (e_ != cudaSuccess) return PSUM_ERR_CUDA;   \
    } while (0)

template <class T>
static int upload(T** dst, const T* src, size_t count) {
    PSUM_CUDA_TRY(cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(count, 1)));
    if (count) PSUM_CUDA_TRY(cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
    return PSUM_OK;
}

// Packs points for the float32 pair kernels: slot i of the pack holds point slot_pt[i]
// (-1: padding far outside the box, never read back), 2 float4 of hi parts per slot
// followed by the same of lo parts, each an offset from its group's float64 origin (the
// centre of the group's bounding box; 4 doubles per group with the radius about it).
static void pack_groups32(const std::vector<double>& pts, const std::vector<int>& slot_pt, int ngroups,
                          std::vector<float4>& pk, std::vector<double>& org) {
    const size_t npk = 2 * (size_t)ngroups * kNearChunk;
    pk.assign(2 * npk, make_float4(0.f, 0.f, 0.f, 0.f));
    for (size_t i = 0; i < npk; ++i) pk[i] = make_float4(1e3f, 1e3f, 1e3f, 1e3f);
    org.assign(4 * (size_t)ngroups, 0.0);
    for (int g = 0; g < ngroups; ++g) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        const int i0 = g * kNearChunk, i1 = (g + 1) * kNearChunk;
        for (int i = i0; i < i1; ++i) {
            if (slot_pt[i] < 0) continue;
            for (int c = 0; c < 3; ++c) {
                lo[c] = std::min(lo[c], pts[3 * (size_t)slot_pt[i] + c]);
                hi[c] = std::max(hi[c], pts[3 * (size_t)slot_pt[i] + c]);
            }
        }
        for (int c = 0; c < 3; ++c) org[4 * g + c] = lo[c] <= hi[c] ? 0.5 * (lo[c] + hi[c]) : 0.0;
        double r2max = 0.0;
        for (int i = i0; i < i1; ++i) {
            if (slot_pt[i] < 0) continue;
            const double* q = &pts[3 * (size_t)slot_pt[i]];
            const double r[3] = {q[0] - org[4 * g], q[1] - org[4 * g + 1], q[2] - org[4 * g + 2]};
            r2max = std::max(r2max, r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            const float f[3] = {(float)r[0], (float)r[1], (float)r[2]};
            const float l[3] = {(float)(r[0] - (double)f[0]), (float)(r[1] - (double)f[1]),
                                (float)(r[2] - (double)f[2])};
            pk[2 * (size_t)i] = make_float4(f[0], f[0], f[1], f[1]);
            pk[2 * (size_t)i + 1] = make_float4(f[2], f[2], 0.f, 0.f);
            pk[npk + 2 * (size_t)i] = make_float4(l[0], l[0], l[1], l[1]);
            pk[npk + 2 * (size_t)i + 1] = make_float4(l[2], l[2], 0.f, 0.f);
        }
        org[4 * g + 3] = std::sqrt(r2max);
    }
}

// The two-layer form of the right-hand side (plans without ball trimming).  The
// partner of y_l is y~_l = y_l - s d_k e_k, so the near block seen from y~_l is the block
// seen from y_l shifted by one period along k: phi_near(y~_l) - phi_near(y_l) is the sum
// over the image layer i_k = s (K_k + 1) minus the sum over the layer i_k = -s K_k (Eq. 3
// at both points; algorithm "get", step 3).  Class c = 2k + (s < 0) fixes the two layers;
// images j < Lmax of a class are its upper layer (weight +1), j >= Lmax its lower layer
// (weight -1), and a class whose layers are smaller than the largest, Lmax, is padded with
// weight-0 entries.  The points are packed class by class in Morton order, float32 plans in
// groups of kNearChunk (tiles of 4 groups), float64 plans in tiles of kTile64 absolute points,
// each point's class in the pack's charge slot (unused for targets).
static int build_check_layers(Plan& pl, const double d[3]) {
    const bool fp32 = pl.opt.precision != PSUM_FP64;
    const int M = pl.opt.M;
    const int* K = pl.opt.K;
    int Lsize[3], Lmax = 0;
    for (int k = 0; k < 3; ++k) {
        Lsize[k] = (2 * K[(k + 1) % 3] + 1) * (2 * K[(k + 2) % 3] + 1);
        Lmax = std::max(Lmax, Lsize[k]);
    }
    const int n_img = 2 * Lmax;
    std::vector<double> sh(6 * (size_t)n_img * 3, 0.0);
    std::vector<float> w(6 * (size_t)n_img, 0.f);
    for (int c = 0; c < 6; ++c) {
        const int k = c / 2, s = (c & 1) ? -1 : 1;
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        for (int side = 0; side < 2; ++side) {
            const int ik = side == 0 ? s * (K[k] + 1) : -s * K[k];
            int j = 0;
            for (int ia = -K[a]; ia <= K[a]; ++ia)
                for (int ib = -K[b]; ib <= K[b]; ++ib, ++j) {
                    double* v = &sh[3 * ((size_t)c * n_img + side * Lmax + j)];
                    v[k] = ik * d[k];
                    v[a] = ia * d[a];
                    v[b] = ib * d[b];
                    w[(size_t)c * n_img + side * Lmax + j] = side == 0 ? 1.f : -1.f;
                }
            for (; j < Lmax; ++j) {   // padding: any finite far image, weight 0
                double* v = &sh[3 * ((size_t)c * n_img + side * Lmax + j)];
                v[k] = ik * d[k];
            }
        }
    }
    // class of each check point from its partner
    std::vector<int> cls(M);
    for (int l = 0; l < M; ++l) {
        int c = -1;
        for (int k = 0; k < 3; ++k) {
            const double dy = pl.Y[3 * (size_t)l + k] - pl.Yt[3 * (size_t)l + k];
            if (dy != 0.0) c = 2 * k + (dy < 0.0 ? 1 : 0);
        }
        if (c < 0) return PSUM_ERR_ARG;     // a partner equal to its point cannot occur on the sphere
        cls[l] = c;
    }
    // class by class, Morton order within a class, each class in whole groups
    std::vector<int> order(M);
    std::iota(order.begin(), order.end(), 0);
    std::vector<uint64_t> key(M);
    for (int l = 0; l < M; ++l) key[l] = morton_host(&pl.Y[3 * (size_t)l], pl.R0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return cls[x] != cls[y] ? cls[x] < cls[y] : key[x] < key[y];
    });
    // one class per target: the points go class by class without padding (a group at a class
    // boundary holds two), the class in the pack's unused charge slot
    std::vector<int> slot(order);
    while (slot.size() % (fp32 ? kTile32 : kTile64)) slot.push_back(-1);
    const int tiles = (int)(slot.size() / (fp32 ? kTile32 : kTile64));
    // the automatic choice takes the layers only where they need no more (target tile, image)
    // units than the points
    if (pl.opt.check_form == PSUM_CHECKS_AUTO && (int64_t)tiles * n_img > (int64_t)pl.n_check_tiles * pl.n_images)
        return PSUM_OK;
    // float32: the kernel keeps an offset per (image, group, class) in shared memory; blocks
    // with K = 3 along two axes would need more than it takes without opt-in
    if (fp32 && near32_dyn_smem(n_img, false, false, kCheckClasses) > kNear32DynSmemMax) return PSUM_OK;
    std::vector<int> pos(M);
    for (size_t i = 0; i < slot.size(); ++i)
        if (slot[i] >= 0) pos[slot[i]] = (int)i;
    int s1;
    if (fp32) {
        std::vector<float4> pk;
        std::vector<double> org;
        pack_groups32(pl.Y, slot, (int)(slot.size() / kNearChunk), pk, org);
        const size_t ng = slot.size() / kNearChunk;
        std::vector<int> gmask(ng, 0);   // classes present in each group
        std::vector<int> npts(ng, 0);
        int last = cls[slot[0]];         // slot 0 holds a point: M >= 1
        for (size_t i = 0; i < slot.size(); ++i) {
            // a padding slot takes the class of the last point before it, which its group
            // holds unless the whole group is padding (it then holds that class alone)
            const int c = slot[i] >= 0 ? cls[slot[i]] : last;
            last = c;
            pk[2 * i + 1].z = (float)c;
            pk[2 * i + 1].w = (float)c;
            gmask[i / kNearChunk] |= 1 << c;
            if (slot[i] >= 0) ++npts[i / kNearChunk];
        }
        // a group of padding alone is marked (kGroupEmpty): the kernel skips a packed target
        // pair of two such groups
        for (size_t g = 0; g < ng; ++g)
            if (!npts[g]) gmask[g] |= kGroupEmpty;
        // per (group, class): centre and radius of the class's points in the group, for the
        // near-unit test (a group at a class boundary spans two caps of the sphere)
        std::vector<double> sub(ng * kCheckClasses * 4, 0.0);
        for (size_t g = 0; g < ng; ++g)
            for (int c = 0; c < kCheckClasses; ++c) {
                double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
                for (size_t i = g * kNearChunk; i < (g + 1) * kNearChunk; ++i)
                    if (slot[i] >= 0 && cls[slot[i]] == c)
                        for (int k = 0; k < 3; ++k) {
                            lo[k] = std::min(lo[k], pl.Y[3 * (size_t)slot[i] + k]);
                            hi[k] = std::max(hi[k], pl.Y[3 * (size_t)slot[i] + k]);
                        }
                double* o = &sub[4 * (g * kCheckClasses + c)];
                if (!(lo[0] <= hi[0])) {      // class absent: the group's own sphere
                    for (int k = 0; k < 4; ++k) o[k] = org[4 * g + k];
                    continue;
                }
                double r2 = 0.0;
                for (int k = 0; k < 3; ++k) o[k] = 0.5 * (lo[k] + hi[k]);
                for (size_t i = g * kNearChunk; i < (g + 1) * kNearChunk; ++i)
                    if (slot[i] >= 0 && cls[slot[i]] == c) {
                        const double* y = &pl.Y[3 * (size_t)slot[i]];
                        r2 = std::max(r2, (y[0] - o[0]) * (y[0] - o[0]) + (y[1] - o[1]) * (y[1] - o[1]) +
                                              (y[2] - o[2]) * (y[2] - o[2]));
                    }
                o[3] = std::sqrt(r2);
            }
        if ((s1 = upload((float4**)&pl.d_lc_tgt, pk.data(), pk.size()))) return s1;
        if ((s1 = upload(&pl.d_lc_org, org.data(), org.size()))) return s1;
        if ((s1 = upload(&pl.d_lc_gmask, gmask.data(), gmask.size()))) return s1;
        if ((s1 = upload(&pl.d_lc_sub, sub.data(), sub.size()))) return s1;
    } else {
        std::vector<double4_32a> pk(slot.size(), make_double4_32a(1e3, 1e3, 1e3, 0.0));
        for (size_t i = 0; i < slot.size(); ++i)
            if (slot[i] >= 0)
                pk[i] = make_double4_32a(pl.Y[3 * (size_t)slot[i]], pl.Y[3 * (size_t)slot[i] + 1],
                                         pl.Y[3 * (size_t)slot[i] + 2], (double)cls[slot[i]]);
        if ((s1 = upload((double4_32a**)&pl.d_lc_tgt, pk.data(), pk.size()))) return s1;
    }
    if ((s1 = upload(&pl.d_lc_pos, pos.data(), pos.size()))) return s1;
    if ((s1 = upload(&pl.d_lc_shifts, sh.data(), sh.size()))) return s1;
    if ((s1 = upload(&pl.d_lc_w, w.data(), w.size()))) return s1;
    pl.lc_tiles = tiles;
    pl.lc_img = n_img;
    if (!fp32) return PSUM_OK;
    // the backward's check sources as the two layers (float32 packing): set (c, side) holds the
    // points of class c, side 0 with the upper layer (weight +1), side 1 with the lower (-1);
    // the source sees the target through the negated image vector
    std::vector<int> bk_slot, bk_img0, bk_nimg;
    std::vector<int> slot_pt;
    for (int c = 0; c < 6; ++c)
        for (int side = 0; side < 2; ++side) {
            std::vector<int> pts;   // Morton order within the class: compact chunks
            for (int l : order)
                if (cls[l] == c) pts.push_back(l);
            if (pts.empty()) continue;
            const int chunks = (int)((pts.size() + kNearChunk - 1) / kNearChunk);
            for (int ch = 0; ch < chunks; ++ch) {
                bk_img0.push_back((2 * c + side) * Lmax);
                bk_nimg.push_back(Lsize[c / 2]);
                for (int k = 0; k < kNearChunk; ++k) {
                    const size_t i = (size_t)ch * kNearChunk + k;
                    bk_slot.push_back(i < pts.size() ? 2 * pts[i] + side : -1);
                    slot_pt.push_back(i < pts.size() ? pts[i] : -1);
                }
            }
        }
    std::vector<double> bsh(12 * (size_t)Lmax * 3, 0.0);
    for (int c = 0; c < 6; ++c)
        for (int side = 0; side < 2; ++side)
            for (int j = 0; j < Lmax; ++j)
                for (int k = 0; k < 3; ++k)
                    bsh[3 * ((size_t)(2 * c + side) * Lmax + j) + k] = -sh[3 * ((size_t)c * n_img + side * Lmax + j) + k];
    const int bk_chunks = (int)bk_img0.size();
    std::vector<float4> bpk;
    std::vector<double> borg;
    pack_groups32(pl.Y, slot_pt, bk_chunks, bpk, borg);
    if ((s1 = upload((float4**)&pl.d_bk_pk, bpk.data(), bpk.size()))) return s1;
    if ((s1 = upload(&pl.d_bk_org, borg.data(), borg.size()))) return s1;
    if ((s1 = upload(&pl.d_bk_slot, bk_slot.data(), bk_slot.size()))) return s1;
    if ((s1 = upload(&pl.d_bk_img0, bk_img0.data(), bk_img0.size()))) return s1;
    if ((s1 = upload(&pl.d_bk_nimg, bk_nimg.data(), bk_nimg.size()))) return s1;
    if ((s1 = upload(&pl.d_bk_shifts, bsh.data(), bsh.size()))) return s1;
    pl.bk_chunks = bk_chunks;
    pl.bk_lmax = Lmax;
    return PSUM_OK;
}

int build_plan(const psum_opts& o, Plan& pl) {
    pl.opt = o;
    const int p = o.p, M = o.M;
    const bool rbf = o.basis == PSUM_BASIS_RBF;
    pl.P = rbf ? o.n_rbf + 1 : (p + 1) * (p + 1);
    const double d[3] = {o.d[0], o.d[1], o.d[2]};
    pl.R0 = 0.5 * std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);             // step 1
    // image vectors of the near block and lambda_eff
    pl.Rb = o.lambda > 0.0 ? o.lambda * pl.R0 : 0.0;
    int K[3] = {o.K[0], o.K[1], o.K[2]};
    if (pl.Rb > 0.0)   // the smallest block that covers the ball S_b
        for (int k = 0; k < 3; ++k) pl.opt.K[k] = K[k] = (int)std::ceil(pl.Rb / d[k] + 0.5);
    pl.shifts.clear();
    pl.self_image = -1;
    for (int i1 = -K[0]; i1 <= K[0]; ++i1)
        for (int i2 = -K[1]; i2 <= K[1]; ++i2)
            for (int i3 = -K[2]; i3 <= K[2]; ++i3) {
                const double p0 = i1 * d[0], p1 = i2 * d[1], p2 = i3 * d[2];
                // with the ball, an image box farther than Rb + R0 holds no kept source
                // (every source lies in the box, within R0 of its centre)
                if (pl.Rb > 0.0 && std::sqrt(p0 * p0 + p1 * p1 + p2 * p2) > (pl.Rb + pl.R0) * (1.0 + 1e-12))
                    continue;
                if (i1 == 0 && i2 == 0 && i3 == 0) pl.self_image = (int)(pl.shifts.size() / 3);
                pl.shifts.push_back(p0);
                pl.shifts.push_back(p1);
                pl.shifts.push_back(p2);
            }
    pl.n_images = (int)(pl.shifts.size() / 3);
    if (pl.n_images > kMaxImages) return PSUM_ERR_ARG;
    double hmin = 1e300;
    for (int k = 0; k < 3; ++k) hmin = std::min(hmin, 0.5 * (2 * K[k] + 1) * d[k]);
    // the ball's radius is the distance to the nearest far-field source
    pl.lambda_eff = pl.Rb > 0.0 ? o.lambda : hmin / pl.R0;

    if (o.points == PSUM_POINTS_GAUSS) {                                              // step 2
        // Gauss spherical grid (Sec. 2.2): polar angles at the zeros of P_{p+1}(cos theta),
        // 2p+1 equispaced azimuths starting at 0
        std::vector<double> t, w;
        gauss_legendre(p + 1, t, w);
        pl.Y.resize(3 * (size_t)M);
        int l = 0;
        for (int i = 0; i <= p; ++i) {
            const double st = std::sqrt(std::max(0.0, 1.0 - t[i] * t[i]));
            for (int j = 0; j < 2 * p + 1; ++j, ++l) {
                const double az = 2.0 * M_PI * j / (2 * p + 1);
                pl.Y[3 * l] = pl.R0 * st * std::cos(az);
                pl.Y[3 * l + 1] = pl.R0 * st * std::sin(az);
                pl.Y[3 * l + 2] = pl.R0 * t[i];
            }
        }
    } else {
        fibonacci_sphere(M, pl.R0, pl.Y);
    }
    partners(pl.Y, d, pl.Yt);                                                         // step 3
    const int n = pl.P - 1;                                                           // step 4
    std::vector<double> A((size_t)M * n);
    if (rbf) {
        // Eq. 5: R_t(y) = 1/|y - x_t| with the centres on a Fibonacci lattice outside S_b
        const double Rs = (o.rbf_radius > 0.0 ? o.rbf_radius : pl.lambda_eff) * pl.R0;
        fibonacci_sphere(n, Rs, pl.Xs);
        auto kern = [&](const double* y, const double* c) {
            const double a = y[0] - c[0], b = y[1] - c[1], e = y[2] - c[2];
            return 1.0 / std::sqrt(a * a + b * b + e * e);
        };
        for (int t = 0; t < n; ++t)
            for (int l = 0; l < M; ++l)
                A[(size_t)t * M + l] = kern(&pl.Y[3 * l], &pl.Xs[3 * t]) - kern(&pl.Yt[3 * l], &pl.Xs[3 * t]);
    } else {
        std::vector<double> b1(pl.P), b2(pl.P);
        const double s = 1.0 / pl.R0;
        for (int l = 0; l < M; ++l) {
            basis_values(pl.Y[3 * l] * s, pl.Y[3 * l + 1] * s, pl.Y[3 * l + 2] * s, p, b1.data());
            basis_values(pl.Yt[3 * l] * s, pl.Yt[3 * l + 1] * s, pl.Yt[3 * l + 2] * s, p, b2.data());
            for (int t = 1; t < pl.P; ++t) A[(size_t)(t - 1) * M + l] = b1[t] - b2[t];
        }
    }
    // the geometry's fingerprint: a stored factorisation is only taken for the same A
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](const std::vector<double>& v) {
        for (double x : v) {
            uint64_t b;
            std::memcpy(&b, &x, sizeof b);
            for (int k = 0; k < 8; ++k) {
                h ^= (b >> (8 * k)) & 0xffu;
                h *= 1099511628211ull;
            }
        }
    };
    mix(pl.Y);
    mix(pl.Yt);
    mix(pl.Xs);
    pl.geom_hash = h;
    int st = PSUM_OK;
    if (!pl.preset_pinv.empty()) {                                                    // step 5, stored
        if (pl.preset_geom != pl.geom_hash || pl.preset_pinv.size() != (size_t)n * M) return PSUM_ERR_IO;
        pl.pinv = pl.preset_pinv;
        pl.rank = pl.preset_rank;
        pl.cond_est = pl.preset_cond;
        if (pl.rank < n) return PSUM_ERR_RANK;
    } else {
        st = qr_pseudo_inverse(A, M, n, pl.pinv, pl.rank, pl.cond_est);               // step 5
    }
    if (st != PSUM_OK) return st;
    if (rbf) {                                                                        // step 6
        // the box mean of 1/|y - x_t| is the single box's Newtonian potential at x_t over V0
        // (App. C applies to the RBF far field)
        pl.Rbox.assign(pl.P, 0.0);
        pl.Rbox[0] = 1.0;
        const double H[3] = {0.5 * d[0], 0.5 * d[1], 0.5 * d[2]};
        for (int t = 0; t < n; ++t) pl.Rbox[t + 1] = block_potential(&pl.Xs[3 * t], H) / (d[0] * d[1] * d[2]);
    } else {
        const int nq = p / 2 + 1;
        std::vector<double> t, w;
        gauss_legendre(nq, t, w);
        pl.Rbox.assign(pl.P, 0.0);
        std::vector<double> b(pl.P);
        for (int i = 0; i < nq; ++i)
            for (int j = 0; j < nq; ++j)
                for (int k = 0; k < nq; ++k) {
                    basis_values(0.5 * d[0] * t[i] / pl.R0, 0.5 * d[1] * t[j] / pl.R0, 0.5 * d[2] * t[k] / pl.R0,
                                 p, b.data());
                    const double ww = w[i] * w[j] * w[k] / 8.0;
                    for (int q = 0; q < pl.P; ++q) pl.Rbox[q] += ww * b[q];
                }
    }

    // ---- check targets: y_0..y_{M-1}, y~_0..y~_{M-1} ----
    pl.n_check = 2 * M;
    std::vector<double> pts(3 * (size_t)pl.n_check);
    std::copy(pl.Y.begin(), pl.Y.end(), pts.begin());
    std::copy(pl.Yt.begin(), pl.Yt.end(), pts.begin() + 3 * (size_t)M);
    std::vector<int> pos(pl.n_check);
    if (o.precision != PSUM_FP64) {   // FP32C and FF: float32 hi/lo packing
        const int tile = kTile32;
        pl.check_tile = tile;
        pl.n_check_tiles = (pl.n_check + tile - 1) / tile;
        const int ngroups = pl.n_check_tiles * kTgt32;
        std::vector<int> order(pl.n_check);
        std::iota(order.begin(), order.end(), 0);
        std::vector<uint64_t> key(pl.n_check);
        for (int j = 0; j < pl.n_check; ++j) key[j] = morton_host(&pts[3 * (size_t)j], pl.R0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
        order.resize((size_t)ngroups * kNearChunk, -1);
        std::vector<float4> pk;
        std::vector<double> org;
        pack_groups32(pts, order, ngroups, pk, org);
        for (size_t i = 0; i < order.size(); ++i)
            if (order[i] >= 0) pos[order[i]] = (int)i;
        std::vector<int> inv((size_t)ngroups * kNearChunk, -1);
        for (int j = 0; j < pl.n_check; ++j) inv[pos[j]] = j;
        int s1 = upload((float4**)&pl.d_check_tgt, pk.data(), pk.size());
        if (s1) return s1;
        s1 = upload(&pl.d_check_org, org.data(), org.size());
        if (s1) return s1;
        s1 = upload(&pl.d_check_inv, inv.data(), inv.size());
        if (s1) return s1;
    } else {
        const int tile = kTile64;
        pl.check_tile = tile;
        pl.n_check_tiles = (pl.n_check + tile - 1) / tile;
        std::vector<double4_32a> pk((size_t)pl.n_check_tiles * tile, make_double4_32a(1e3, 1e3, 1e3, 0.0));
        for (int j = 0; j < pl.n_check; ++j) {
            pk[j] = make_double4_32a(pts[3 * (size_t)j], pts[3 * (size_t)j + 1], pts[3 * (size_t)j + 2], 0.0);
            pos[j] = j;
        }
        int s1 = upload((double4_32a**)&pl.d_check_tgt, pk.data(), pk.size());
        if (s1) return s1;
    }
    int s2 = upload(&pl.d_check_pos, pos.data(), pos.size());
    if (s2) return s2;
    pl.lc_tiles = 0;
    pl.lc_img = 0;
    if (!(pl.Rb > 0.0) && o.check_form != PSUM_CHECKS_POINTS && (s2 = build_check_layers(pl, d)))
        return s2;
    if ((s2 = upload(&pl.d_pinv, pl.pinv.data(), pl.pinv.size()))) return s2;
    if ((s2 = upload(&pl.d_Rbox, pl.Rbox.data(), pl.Rbox.size()))) return s2;
    if ((s2 = upload(&pl.d_shifts, pl.shifts.data(), pl.shifts.size()))) return s2;
    if (rbf && (s2 = upload(&pl.d_rbf, pl.Xs.data(), pl.Xs.size()))) return s2;
    {
        std::vector<double> tab(sh_tab_size(p));
        sh_tab_fill(p, tab.data());
        std::vector<float> tabf(tab.begin(), tab.end());
        if ((s2 = upload(&pl.d_shtab64, tab.data(), tab.size()))) return s2;
        if ((s2 = upload(&pl.d_shtab32, tabf.data(), tabf.size()))) return s2;
    }
    PSUM_CUDA_TRY(cudaMalloc((void**)&pl.d_C, sizeof(double) * pl.P));
    PSUM_CUDA_TRY(cudaMemset(pl.d_C, 0, sizeof(double) * pl.P));
    PSUM_CUDA_TRY(cudaMalloc((void**)&pl.d_status, sizeof(int)));
    PSUM_CUDA_TRY(cudaMemset(pl.d_status, 0, sizeof(int)));
    PSUM_CUDA_TRY(cudaMallocHost((void**)&pl.h_status, sizeof(int)));
    *pl.h_status = 0;
    return PSUM_OK;
}

void free_plan_device(Plan& pl) {
    cudaFree(pl.d_check_pos);
    cudaFree(pl.d_check_inv);
    cudaFree(pl.d_check_tgt);
    cudaFree(pl.d_check_org);
    cudaFree(pl.d_lc_tgt);
    cudaFree(pl.d_lc_org);
    cudaFree(pl.d_lc_gmask);
    cudaFree(pl.d_lc_sub);
    cudaFree(pl.d_lc_pos);
    cudaFree(pl.d_lc_shifts);
    cudaFree(pl.d_lc_w);
    cudaFree(pl.d_bk_pk);
    cudaFree(pl.d_bk_org);
    cudaFree(pl.d_bk_slot);
    cudaFree(pl.d_bk_img0);
    cudaFree(pl.d_bk_nimg);
    cudaFree(pl.d_bk_shifts);
    cudaFree(pl.d_pinv);
    cudaFree(pl.d_Rbox);
    cudaFree(pl.d_shifts);
    cudaFree(pl.d_rbf);
    cudaFree(pl.d_shtab64);
    cudaFree(pl.d_shtab32);
    cudaFree(pl.d_C);
    cudaFree(pl.d_status);
    if (pl.h_status) cudaFreeHost(pl.h_status);
    cudaFree(pl.scratch.ptr);
    cudaFree(pl.dstage.ptr);
    pl = Plan();
}

}  // namespace psum
