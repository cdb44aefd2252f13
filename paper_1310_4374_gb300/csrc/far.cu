// Everything in algorithm "get" (Sec. 2.3.2) around the near-field sum:
//   validation (Eq. 1: neutral box, positions inside it),
//   the right-hand side f and the least-squares coefficients (steps 4-5, Eqs. 8-10),
//   the constant C_1 from the zero-mean condition (step 6, Eqs. pfx3-pfx4, App. C),
//   the far field and its gradient at the charges and the final sum (steps 7-8,
//   Eqs. 1.6-1.9).
// All of it runs in float64.
#include "psum_internal.cuh"
#include "mean.cuh"

namespace psum {

// ---------------------------------------------------------------------------
// block reduction of two doubles (fixed order for a fixed block size)
// ---------------------------------------------------------------------------
template <int BS>
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[BS / 32], sb[BS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        a = l < BS / 32 ? sa[l] : 0.0;
        b = l < BS / 32 ? sb[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

constexpr int kRedThreads = 256;

// Eq. 1: charges must sum to zero; positions must lie in [-d/2, d/2).
__global__ void __launch_bounds__(kRedThreads) k_validate(const double* __restrict__ x, const double* __restrict__ q,
                                                          int64_t n, double d0, double d1, double d2,
                                                          double* __restrict__ partial, int* __restrict__ status) {
    double s = 0.0, sa = 0.0;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
        const double a = x[3 * i], b = x[3 * i + 1], c = x[3 * i + 2], qi = q[i];
        const bool in = (a >= -0.5 * d0) && (a < 0.5 * d0) && (b >= -0.5 * d1) && (b < 0.5 * d1) &&
                        (c >= -0.5 * d2) && (c < 0.5 * d2);
        if (!in) bad |= kStatOutOfBox;           // also catches NaN positions
        if (!(fabs(qi) <= 1.7976931348623157e308)) bad |= kStatNonFinite;
        s += qi;
        sa += fabs(qi);
    }
    if (bad) atomicOr(status, bad);
    block_sum2<kRedThreads>(s, sa);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s;
        partial[2 * blockIdx.x + 1] = sa;
    }
}

// Evaluation points: inside the half-open box and finite, like the charges.
__global__ void __launch_bounds__(kRedThreads) k_validate_points(const double* __restrict__ y, int64_t n, double d0,
                                                                 double d1, double d2, int* __restrict__ status) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
        const double a = y[3 * i], b = y[3 * i + 1], c = y[3 * i + 2];
        const bool in = (a >= -0.5 * d0) && (a < 0.5 * d0) && (b >= -0.5 * d1) && (b < 0.5 * d1) &&
                        (c >= -0.5 * d2) && (c < 0.5 * d2);
        if (!in) bad |= kStatOutOfBox;
    }
    if (bad) atomicOr(status, bad);
}

__global__ void k_validate_finish(const double* __restrict__ partial, int nblk, int* __restrict__ status) {
    double s = 0.0, sa = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) { s += partial[2 * b]; sa += partial[2 * b + 1]; }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        sa += __shfl_down_sync(0xffffffffu, sa, o);
    }
    if (threadIdx.x == 0 && !(fabs(s) <= 1e-12 * sa)) atomicOr(status, kStatNonNeutral);
}

// One (charge, term) pair per work item: sum_i q_i U(x_i) with U the regrouped corner sum
// over the block (12 terms, each one logarithm and one two-argument arctangent; every charge
// of the box lies inside the block).  Twelve items per
// charge in blocks of 64 threads keep small systems from running a handful of blocks through
// the float64 pipes of a few SMs (4000 charges: 148 us with one 256-thread block per 256
// charges).
constexpr int kMeanThreads = 64;
constexpr int kMeanTerms = 12;

__global__ void __launch_bounds__(kMeanThreads) k_box_mean(const double* __restrict__ x, const double* __restrict__ q,
                                                           int64_t n, double H0, double H1, double H2,
                                                           double* __restrict__ partial) {
    const double H[3] = {H0, H1, H2};
    double s = 0.0, dummy = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * kMeanThreads + threadIdx.x; k < kMeanTerms * n;
         k += (int64_t)gridDim.x * kMeanThreads) {
        const int64_t i = k / kMeanTerms;
        const int j = (int)(k - i * kMeanTerms);
        const double X[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        s += q[i] * box_potential_paired_term(X, H, j);
    }
    block_sum2<kMeanThreads>(s, dummy);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// With the near set trimmed to the ball S_b (get step 2) every kept source image x + p
// (|x + p| <= Rb, the same float64 test as the pair kernels) contributes the potential of the
// box at x + p.  Along a line of images (fixed offsets on axes 0 and 1) the kept ones come in
// runs, and a run of boxes is one rod-shaped box: its potential is one regrouped corner sum
// (12 logarithms, 12 arctangents) instead of one per box.  The covering block's lattice is
// walked directly (i d_k is the image table's float64 value), so every kept test matches the
// pair kernels'.  Which images are kept depends on the charge, so the threads of a warp take
// charges in Hilbert order when a permutation is given: neighbours see nearly the same runs.
__global__ void __launch_bounds__(kRedThreads) k_box_mean_ball(const double* __restrict__ x,
                                                               const double* __restrict__ q,
                                                               const uint32_t* __restrict__ perm, int64_t n,
                                                               double d0, double d1, double d2, int K0, int K1,
                                                               int K2, double Rb, double* __restrict__ partial) {
    const double Rb2 = __dmul_rn(Rb, Rb);
    double s = 0.0, dummy = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kRedThreads) {
        const int64_t i = perm ? (int64_t)perm[k] : k;
        const double x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        double u = 0.0;
        for (int i1 = -K0; i1 <= K0; ++i1) {
            const double a = __dadd_rn(x0, i1 * d0);
            for (int i2 = -K1; i2 <= K1; ++i2) {
                const double b = __dadd_rn(x1, i2 * d1);
                const double ab = __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b));
                if (ab > Rb2) continue;            // c^2 >= 0: no image of this line is kept
                int lo = 0;
                bool run = false;
                for (int i3 = -K2; i3 <= K2 + 1; ++i3) {
                    bool kept = false;
                    if (i3 <= K2) {
                        const double c = __dadd_rn(x2, i3 * d2);
                        kept = __dadd_rn(ab, __dmul_rn(c, c)) <= Rb2;
                    }
                    if (kept && !run) {
                        lo = i3;
                        run = true;
                    } else if (!kept && run) {
                        // the run lo .. i3 - 1: one box of i3 - lo images along axis 2
                        const double X[3] = {a, b, x2 + 0.5 * (double)(lo + i3 - 1) * d2};
                        const double H[3] = {0.5 * d0, 0.5 * d1, 0.5 * (double)(i3 - lo) * d2};
                        u += box_potential_paired(X, H);
                        run = false;
                    }
                }
            }
        }
        s += q[i] * u;
    }
    block_sum2<kRedThreads>(s, dummy);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Steps 4-5: f_l = phi_near(y~_l) - phi_near(y_l), C_{2..P} = A^+ f.
// One warp per row of the (P-1) x M pseudo-inverse.
// ---------------------------------------------------------------------------
constexpr int kProjThreads = 256;

// f_l = phi_near(y~_l) - phi_near(y_l); with `layers` the check sums already hold the
// difference (the two image layers at y_l), at packed position check_pos[l].
__global__ void k_rhs(const double* __restrict__ phi_check, const int* __restrict__ check_pos, int M,
                      int layers, double* __restrict__ f) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < M) f[l] = layers ? phi_check[check_pos[l]] : phi_check[check_pos[M + l]] - phi_check[check_pos[l]];
}

__global__ void __launch_bounds__(kProjThreads) k_project(const double* __restrict__ pinv, int rows, int M,
                                                          const double* __restrict__ f, double* __restrict__ C) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (kProjThreads / 32) + w;
    if (row >= rows) return;
    const double* a = pinv + (int64_t)row * M;
    double s = 0.0;
    for (int l = lane; l < M; l += 32) s = fma(a[l], f[l], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) C[1 + row] = s;
}

// Step 6 (Eq. pfx3 with phi_mean = 0): C_1 = -<phi_near> - sum_{t>=2} C_t R_t^(0).
__global__ void k_constant(double* __restrict__ C, const double* __restrict__ Rbox, int P,
                           const double* __restrict__ mean_partial, int nblk, double inv_V0, int zero_mean) {
    double s = 0.0, m = 0.0;
    if (zero_mean) {
        for (int t = 1 + threadIdx.x; t < P; t += 32) s = fma(C[t], Rbox[t], s);
        for (int b = threadIdx.x; b < nblk; b += 32) m += mean_partial[b];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        m += __shfl_down_sync(0xffffffffu, m, o);
    }
    if (threadIdx.x == 0) C[0] = zero_mean ? (-m * inv_V0 - s) : 0.0;
}

// ---------------------------------------------------------------------------
// Steps 7-8: phi = phi_near + C_1 + sum_t C_t R_t(x/R0), grad likewise
// (the gradient of the expansion by differentiating the recurrence), written
// back to the caller's order.
// ---------------------------------------------------------------------------
constexpr int kFarThreads = 128;

// T = double for FP64 plans; T = float for FP32C plans, whose far field is a smooth,
// slowly varying part of phi (its float32 evaluation errors sit well below the pair sum's)
template <class T>
__global__ void __launch_bounds__(kFarThreads) k_far_combine(const double* __restrict__ x, int64_t n,
                                                             const int* __restrict__ perm,
                                                             const double* __restrict__ phi_near,
                                                             const double* __restrict__ grad_near,
                                                             const double* __restrict__ C, int p, double inv_R0,
                                                             const T* __restrict__ tab,
                                                             const int* __restrict__ status,
                                                             double* __restrict__ phi, double* __restrict__ grad,
                                                             int* __restrict__ status_out) {
    extern __shared__ unsigned char s_raw[];
    const int P = (p + 1) * (p + 1);
    const int nt = sh_tab_size(p);
    T* s_C = (T*)s_raw;
    T* s_tab = s_C + P;
    for (int t = threadIdx.x; t < P; t += kFarThreads) s_C[t] = (T)C[t];
    for (int t = threadIdx.x; t < nt; t += kFarThreads) s_tab[t] = tab[t];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * kFarThreads + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm ? (int64_t)perm[s] : s;
    const bool failed = (*status & (kStatNonNeutral | kStatOutOfBox | kStatNonFinite | kStatTimeout | kStatBounds)) != 0;
    if (failed) {
        phi[i] = __longlong_as_double(0x7ff8000000000000ll);
        if (grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const T ux = (T)(x[3 * i] * inv_R0), uy = (T)(x[3 * i + 1] * inv_R0), uz = (T)(x[3 * i + 2] * inv_R0);
    T f = 0, gx = 0, gy = 0, gz = 0;
    if (grad) {
        sh_visit_tab<true>(ux, uy, uz, p, s_tab, [&](int nn, int mm, T v, T vx, T vy, T vz) {
            const T c = s_C[sh_index(nn, mm)];
            f = fma(c, v, f);
            gx = fma(c, vx, gx);
            gy = fma(c, vy, gy);
            gz = fma(c, vz, gz);
        });
    } else {
        sh_visit_tab<false>(ux, uy, uz, p, s_tab, [&](int nn, int mm, T v, T, T, T) {
            f = fma(s_C[sh_index(nn, mm)], v, f);
        });
    }
    // the t = 1 term of the sum is C_1 R^_0^0 = C_1: included by the visitor
    const double ph = phi_near[s] + (double)f;
    phi[i] = ph;
    bool finite = fabs(ph) <= 1.7976931348623157e308;
    if (grad) {
        const double g0 = grad_near[3 * s] + (double)gx * inv_R0;
        const double g1 = grad_near[3 * s + 1] + (double)gy * inv_R0;
        const double g2 = grad_near[3 * s + 2] + (double)gz * inv_R0;
        grad[3 * i] = g0;
        grad[3 * i + 1] = g1;
        grad[3 * i + 2] = g2;
        finite = finite && fabs(g0) <= 1.7976931348623157e308 && fabs(g1) <= 1.7976931348623157e308 &&
                 fabs(g2) <= 1.7976931348623157e308;
    }
    if (!finite) atomicOr(status_out, kStatNonFinite);
}

// Steps 7-8 with the RBF basis of Eq. 5: phi_far(y) = C_1 + sum_t C_{t+1} / |y - x_t| and
// its gradient, a pair sum of the targets against the n_rbf centres in float64 (the
// least-squares coefficients of kernel functions cancel strongly: a float32 sum would
// lose digits to that cancellation).  Centres with their coefficients are staged in
// shared memory in blocks of kRbfBlock.
constexpr int kRbfBlock = 256;

template <bool kGrad>
__global__ void __launch_bounds__(kFarThreads) k_far_rbf(const double* __restrict__ x, int64_t n,
                                                         const int* __restrict__ perm,
                                                         const double* __restrict__ phi_near,
                                                         const double* __restrict__ grad_near,
                                                         const double* __restrict__ C,
                                                         const double* __restrict__ centres, int S,
                                                         const int* __restrict__ status,
                                                         double* __restrict__ phi, double* __restrict__ grad,
                                                         int* __restrict__ status_out) {
    __shared__ double4_32a s_c[kRbfBlock];
    const int64_t s = (int64_t)blockIdx.x * kFarThreads + threadIdx.x;
    const bool live = s < n;
    const int64_t i = live ? (perm ? (int64_t)perm[s] : s) : 0;
    const double y0 = live ? x[3 * i] : 0.0, y1 = live ? x[3 * i + 1] : 0.0, y2 = live ? x[3 * i + 2] : 0.0;
    double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int t0 = 0; t0 < S; t0 += kRbfBlock) {
        const int nb = S - t0 < kRbfBlock ? S - t0 : kRbfBlock;
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += kFarThreads) {
            const double* c = centres + 3 * (size_t)(t0 + t);
            s_c[t] = make_double4_32a(c[0], c[1], c[2], C[1 + t0 + t]);
        }
        __syncthreads();
        for (int t = 0; t < nb; ++t) {
            const double4_32a c = s_c[t];
            const double a = y0 - c.x, b = y1 - c.y, e = y2 - c.z;
            const double ri = rsqrt(fma(e, e, fma(b, b, a * a)));
            const double cr = c.w * ri;
            f += cr;
            if (kGrad) {
                const double cr3 = cr * ri * ri;
                gx = fma(-cr3, a, gx);
                gy = fma(-cr3, b, gy);
                gz = fma(-cr3, e, gz);
            }
        }
    }
    if (!live) return;
    const bool failed = (*status & (kStatNonNeutral | kStatOutOfBox | kStatNonFinite | kStatTimeout | kStatBounds)) != 0;
    if (failed) {
        phi[i] = __longlong_as_double(0x7ff8000000000000ll);
        if (grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const double ph = phi_near[s] + (C[0] + f);
    phi[i] = ph;
    bool finite = fabs(ph) <= 1.7976931348623157e308;
    if (kGrad) {
        const double g0 = grad_near[3 * s] + gx, g1 = grad_near[3 * s + 1] + gy, g2 = grad_near[3 * s + 2] + gz;
        grad[3 * i] = g0;
        grad[3 * i + 1] = g1;
        grad[3 * i + 2] = g2;
        finite = finite && fabs(g0) <= 1.7976931348623157e308 && fabs(g1) <= 1.7976931348623157e308 &&
                 fabs(g2) <= 1.7976931348623157e308;
    }
    if (!finite) atomicOr(status_out, kStatNonFinite);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_far_rbf(const double* x, int64_t n, const int* perm, const double* phi_near,
                           const double* grad_near, const double* C, const double* centres, int S, const int* status,
                           double* phi, double* grad, int* status_out, cudaStream_t st) {
    const unsigned nb = (unsigned)((n + kFarThreads - 1) / kFarThreads);
    if (grad)
        k_far_rbf<true><<<nb, kFarThreads, 0, st>>>(x, n, perm, phi_near, grad_near, C, centres, S, status, phi,
                                                    grad, status_out);
    else
        k_far_rbf<false><<<nb, kFarThreads, 0, st>>>(x, n, perm, phi_near, grad_near, C, centres, S, status, phi,
                                                     grad, status_out);
    return cudaGetLastError();
}

int reduce_blocks(int64_t n, int num_sms) {
    int64_t nb = (n + kRedThreads - 1) / kRedThreads;
    const int64_t cap = 4LL * num_sms;
    if (nb > cap) nb = cap;
    return nb < 1 ? 1 : (int)nb;
}

cudaError_t launch_validate_points(const double* y, int64_t n, const double d[3], int nblk, int* status,
                                   cudaStream_t st) {
    k_validate_points<<<nblk, kRedThreads, 0, st>>>(y, n, d[0], d[1], d[2], status);
    return cudaGetLastError();
}

cudaError_t launch_validate(const double* x, const double* q, int64_t n, const double d[3], double* partial,
                            int nblk, int* status, cudaStream_t st) {
    k_validate<<<nblk, kRedThreads, 0, st>>>(x, q, n, d[0], d[1], d[2], partial, status);
    k_validate_finish<<<1, 32, 0, st>>>(partial, nblk, status);
    return cudaGetLastError();
}

int mean_blocks(int64_t n, int num_sms) {
    int64_t nb = (kMeanTerms * n + kMeanThreads - 1) / kMeanThreads;
    const int64_t cap = 16LL * num_sms;
    if (nb > cap) nb = cap;
    return nb < 1 ? 1 : (int)nb;
}

cudaError_t launch_box_mean(const double* x, const double* q, int64_t n, const double H[3], double* partial,
                            int nblk, cudaStream_t st) {
    k_box_mean<<<nblk, kMeanThreads, 0, st>>>(x, q, n, H[0], H[1], H[2], partial);
    return cudaGetLastError();
}

cudaError_t launch_box_mean_ball(const double* x, const double* q, const uint32_t* perm, int64_t n,
                                 const double d[3], const int K[3], double Rb, double* partial, int nblk,
                                 cudaStream_t st) {
    k_box_mean_ball<<<nblk, kRedThreads, 0, st>>>(x, q, perm, n, d[0], d[1], d[2], K[0], K[1], K[2], Rb, partial);
    return cudaGetLastError();
}

cudaError_t launch_project(const double* pinv, int rows, int M, const double* phi_check, const int* check_pos,
                           double* f, double* C, cudaStream_t st, bool layers) {
    k_rhs<<<(M + 255) / 256, 256, 0, st>>>(phi_check, check_pos, M, layers ? 1 : 0, f);
    const int per = kProjThreads / 32;
    k_project<<<(rows + per - 1) / per, kProjThreads, 0, st>>>(pinv, rows, M, f, C);
    return cudaGetLastError();
}

cudaError_t launch_constant(double* C, const double* Rbox, int P, const double* mean_partial, int nblk,
                            double inv_V0, int zero_mean, cudaStream_t st) {
    k_constant<<<1, 32, 0, st>>>(C, Rbox, P, mean_partial, nblk, inv_V0, zero_mean);
    return cudaGetLastError();
}

cudaError_t launch_far_combine(const double* x, int64_t n, const int* perm, const double* phi_near,
                               const double* grad_near, const double* C, int p, double inv_R0, const double* tab64,
                               const float* tab32, const int* status, double* phi, double* grad, int* status_out,
                               cudaStream_t st) {
    const int P = (p + 1) * (p + 1);
    const unsigned nb = (unsigned)((n + kFarThreads - 1) / kFarThreads);
    if (tab32) {
        const size_t smem = sizeof(float) * (P + sh_tab_size(p));
        k_far_combine<float><<<nb, kFarThreads, smem, st>>>(x, n, perm, phi_near, grad_near, C, p, inv_R0, tab32,
                                                            status, phi, grad, status_out);
    } else {
        const size_t smem = sizeof(double) * (P + sh_tab_size(p));
        k_far_combine<double><<<nb, kFarThreads, smem, st>>>(x, n, perm, phi_near, grad_near, C, p, inv_R0, tab64,
                                                             status, phi, grad, status_out);
    }
    return cudaGetLastError();
}

}  // namespace psum
