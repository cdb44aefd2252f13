// Energy E = 1/2 sum_j q_j phi(x_j) and its exact derivatives for the discrete method.
//
// phi = phi_near + phi_far, phi_far = C_1 + sum_{t>=2} C_t R_t(x/R0), C_{2..P} = A^+ f and
// f_l = phi_near(y~_l) - phi_near(y_l) is linear in q (Eqs. 3, 8-10).  The adjoint of the
// least-squares fit gives, with the moments w_t = sum_j q_j R_t(x_j/R0) and u = (A^+)^T w,
//   psi(x)   = sum_l u_l [G(y~_l - x) - G(y_l - x)]   (G: the near-block image kernel),
//   dE/dq_k  = phi(x_k) - phi_far(x_k)/2 + psi(x_k)/2,
//   dE/dx_k  = q_k [grad phi - grad phi_far/2 + grad psi/2](x_k).
// psi is a near-field sum of check-point charges at the charges, done by the same pair kernels
// as the forward sum: 2M charges (+u at y~, -u at y) with the near block's images, or, as the
// right-hand side's two image layers, M points twice (+u_l with the upper layer's images, -u_l
// with the lower's; float32 packing with plans that take the layers).
#include "psum_internal.cuh"

namespace psum {

constexpr int kMomThreads = 128;

// phi_far (with C_1) and grad phi_far at every charge, and per-block partial moments.
__global__ void __launch_bounds__(kMomThreads) k_moments(const double* __restrict__ x, const double* __restrict__ q,
                                                         int64_t n, const double* __restrict__ C, int p,
                                                         double inv_R0, const double* __restrict__ tab,
                                                         double* __restrict__ far_phi,
                                                         double* __restrict__ far_grad,
                                                         double* __restrict__ w_partial) {
    extern __shared__ double sm[];
    const int P = (p + 1) * (p + 1);
    constexpr int W = kMomThreads / 32;
    double* s_C = sm;
    double* s_w = sm + P;                                   // [warps][P]
    double* s_tab = s_w + W * P;
    for (int t = threadIdx.x; t < P; t += kMomThreads) s_C[t] = C[t];
    for (int t = threadIdx.x; t < sh_tab_size(p); t += kMomThreads) s_tab[t] = tab[t];
    for (int t = threadIdx.x; t < W * P; t += kMomThreads) s_w[t] = 0.0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kMomThreads + threadIdx.x;
    const bool valid = i < n;
    const double qi = valid ? q[i] : 0.0;
    const double ux = valid ? x[3 * i] * inv_R0 : 0.0;
    const double uy = valid ? x[3 * i + 1] * inv_R0 : 0.0;
    const double uz = valid ? x[3 * i + 2] * inv_R0 : 0.0;
    double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    double* ws = s_w + warp * P;
    sh_visit_tab<true>(ux, uy, uz, p, s_tab, [&](int nn, int mm, double v, double vx, double vy, double vz) {
        const int t = sh_index(nn, mm);
        const double c = s_C[t];
        f = fma(c, v, f);
        gx = fma(c, vx, gx);
        gy = fma(c, vy, gy);
        gz = fma(c, vz, gz);
        double m = qi * v;
        for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
        if (lane == 0) ws[t] += m;
    });
    if (valid) {
        far_phi[i] = f;
        far_grad[3 * i] = gx * inv_R0;
        far_grad[3 * i + 1] = gy * inv_R0;
        far_grad[3 * i + 2] = gz * inv_R0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < P; t += kMomThreads) {
        double s = 0.0;
        for (int w = 0; w < W; ++w) s += s_w[w * P + t];
        w_partial[(int64_t)blockIdx.x * P + t] = s;
    }
}

__global__ void k_moments_reduce(const double* __restrict__ w_partial, int nblk, int P, double* __restrict__ w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += w_partial[(int64_t)b * P + t];
    w[t] = s;
}

// u = (A^+)^T w over the non-constant moments t = 2..P.
__global__ void k_adjoint(const double* __restrict__ pinv, int rows, int M, const double* __restrict__ w,
                          double* __restrict__ u) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= M) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s = fma(pinv[(int64_t)r * M + l], w[1 + r], s);
    u[l] = s;
}

// The check points as sources of psi with charges from u (packed positions from the plan).
// Point form (layers == 0): slot s holds point j = inv[s] (j < M: y_j, charge -u_j; else
// y~_{j-M}, charge +u_{j-M}).  Two-layer form: inv[s] = 2 l + side, charge +u_l with the upper
// layer's images (side 0), -u_l with the lower layer's (side 1).  -1: padding, charge 0.  With
// out_lo (float-float plans) the lo parts are copied too, with the charges' float32 remainders.
__global__ void k_check_sources32(const float4* __restrict__ chk_hi, const float4* __restrict__ chk_lo,
                                  const int* __restrict__ inv, int64_t n_pts, int M, const double* __restrict__ u,
                                  float4* __restrict__ out_hi, float4* __restrict__ out_lo, int layers) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pts) return;
    const int j = inv[s];
    double cd = 0.0;
    if (j >= 0) {
        if (layers)
            cd = (j & 1) ? -u[j >> 1] : u[j >> 1];
        else
            cd = j < M ? -u[j] : u[j - M];
    }
    const float c = (float)cd;
    const float4 A = chk_hi[2 * s], B = chk_hi[2 * s + 1];
    out_hi[2 * s] = A;
    out_hi[2 * s + 1] = make_float4(B.x, B.y, c, c);
    if (out_lo) {
        const float cl = (float)(cd - (double)c);
        const float4 C = chk_lo[2 * s], D = chk_lo[2 * s + 1];
        out_lo[2 * s] = C;
        out_lo[2 * s + 1] = make_float4(D.x, D.y, cl, cl);
    }
}

__global__ void k_check_sources64(const double4_32a* __restrict__ chk, int64_t n_pts, int M,
                                  const double* __restrict__ u, double4_32a* __restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pts) return;
    const double4_32a P = chk[s];
    double c = 0.0;
    if (s < 2 * M) c = s < M ? -u[s] : u[s - M];
    out[s] = make_double4_32a(P.x, P.y, P.z, c);
}

__global__ void k_backward_combine(int64_t n, const int* __restrict__ perm, const double* __restrict__ q,
                                   const double* __restrict__ phi, const double* __restrict__ grad,
                                   const double* __restrict__ far_phi, const double* __restrict__ far_grad,
                                   const double* __restrict__ psi, const double* __restrict__ gpsi,
                                   const double* __restrict__ gE, double* __restrict__ dEdq,
                                   double* __restrict__ dEdx) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm ? (int64_t)perm[s] : s;
    const double g = gE ? *gE : 1.0;
    if (dEdq) dEdq[i] = g * (phi[i] - 0.5 * far_phi[i] + 0.5 * psi[s]);
    if (dEdx) {
        const double qi = g * q[i];
        for (int c = 0; c < 3; ++c)
            dEdx[3 * i + c] = qi * (grad[3 * i + c] - 0.5 * far_grad[3 * i + c] + 0.5 * gpsi[3 * s + c]);
    }
}

// E = 1/2 sum q phi, fixed-order reduction
constexpr int kEnThreads = 256;
__global__ void __launch_bounds__(kEnThreads) k_energy_partial(const double* __restrict__ q,
                                                               const double* __restrict__ phi, int64_t n,
                                                               double* __restrict__ partial) {
    __shared__ double sh[kEnThreads / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kEnThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kEnThreads)
        s = fma(q[i], phi[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kEnThreads / 32; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_energy_finish(const double* __restrict__ partial, int nblk, double* __restrict__ E) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += partial[b];
        *E = 0.5 * t;
    }
}

// ---------------------------------------------------------------------------
size_t moments_smem(int p);

cudaError_t launch_moments(const double* x, const double* q, int64_t n, const double* C, int p, double inv_R0,
                           const double* tab, double* far_phi, double* far_grad, double* w_partial, int nblk,
                           double* w, cudaStream_t st) {
    const int P = (p + 1) * (p + 1);
    const size_t smem = moments_smem(p);
    k_moments<<<nblk, kMomThreads, smem, st>>>(x, q, n, C, p, inv_R0, tab, far_phi, far_grad, w_partial);
    k_moments_reduce<<<(P + 127) / 128, 128, 0, st>>>(w_partial, nblk, P, w);
    return cudaGetLastError();
}

cudaError_t set_moments_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int moments_blocks(int64_t n) { return (int)((n + kMomThreads - 1) / kMomThreads); }

size_t moments_smem(int p) {
    return sizeof(double) * ((p + 1) * (p + 1) * (1 + kMomThreads / 32) + sh_tab_size(p));
}

cudaError_t launch_adjoint(const double* pinv, int rows, int M, const double* w, double* u, cudaStream_t st) {
    k_adjoint<<<(M + 127) / 128, 128, 0, st>>>(pinv, rows, M, w, u);
    return cudaGetLastError();
}

cudaError_t launch_check_sources32(const float4* chk_hi, const float4* chk_lo, const int* inv, int64_t n_pts, int M,
                                   const double* u, float4* out_hi, float4* out_lo, cudaStream_t st, bool layers) {
    k_check_sources32<<<(unsigned)((n_pts + 255) / 256), 256, 0, st>>>(chk_hi, chk_lo, inv, n_pts, M, u, out_hi,
                                                                         out_lo, layers ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_check_sources64(const double4_32a* chk, int64_t n_pts, int M, const double* u,
                                   double4_32a* out, cudaStream_t st) {
    k_check_sources64<<<(unsigned)((n_pts + 255) / 256), 256, 0, st>>>(chk, n_pts, M, u, out);
    return cudaGetLastError();
}

cudaError_t launch_backward_combine(int64_t n, const int* perm, const double* q, const double* phi,
                                    const double* grad, const double* far_phi, const double* far_grad,
                                    const double* psi, const double* gpsi, const double* gE, double* dEdq,
                                    double* dEdx, cudaStream_t st) {
    k_backward_combine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, q, phi, grad, far_phi, far_grad, psi,
                                                                    gpsi, gE, dEdq, dEdx);
    return cudaGetLastError();
}

cudaError_t launch_energy(const double* q, const double* phi, int64_t n, double* partial, int nblk, double* E,
                          cudaStream_t st) {
    k_energy_partial<<<nblk, kEnThreads, 0, st>>>(q, phi, n, partial);
    k_energy_finish<<<1, 32, 0, st>>>(partial, nblk, E);
    return cudaGetLastError();
}

}  // namespace psum
