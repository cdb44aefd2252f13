// Host-side launchers of the device kernels (one definition each in near.cu, sort.cu,
// far.cu, backward.cu, batch.cu).
#pragma once

#include "psum_internal.cuh"

namespace psum {
// near.cu
cudaError_t launch_near32(bool grad, const float4* src_hi, const float4* src_lo, const double* src_org,
                          const float4* tgt_hi, const float4* tgt_lo, const double* tgt_org, const double* shifts,
                          double* partial, const NearPlanLaunch& L, cudaStream_t st, int variant = 0,
                          const double* src_x = nullptr, double Rb = 0.0, bool ff = false,
                          const int* grp_cls = nullptr, const float* img_w = nullptr, int n_cls = 1,
                          const double* grp_sub = nullptr, const int* chunk_img0 = nullptr,
                          const int* chunk_nimg = nullptr);
cudaError_t launch_near64(bool grad, const double4_32a* src, const double4_32a* tgt, const double* shifts,
                          double* partial, const NearPlanLaunch& L, cudaStream_t st, double Rb = 0.0,
                          const float* img_w = nullptr, int n_cls = 1);
constexpr int kCheckClasses = 6;   // two-layer check sums: partner axis and side
// dynamic shared memory of k_near32 for n_img images and n_cls image lists per target group;
// the launches stay within the 48 KiB that needs no opt-in
size_t near32_dyn_smem(int n_img, bool trimmed, bool grad, int n_cls);
constexpr size_t kNear32DynSmemMax = 48 * 1024;
cudaError_t launch_near_reduce(const double* partial, int64_t n_valid, int tile_size, int nq,
                               const NearPlanLaunch& L, double* out_phi, double* out_grad, cudaStream_t st);
int near32_occupancy_ctas(int n_img, int variant = 0, bool trimmed = false, bool ff = false, bool grad = true,
                          int n_cls = 1);
// register budget of the check-point (potential-only) launch of block plans: 0 = 4 CTAs/SM, 1 = 6
#ifndef PSUM_CHECK_VARIANT
#define PSUM_CHECK_VARIANT 0
#endif
constexpr int kCheckVariant = PSUM_CHECK_VARIANT;
cudaError_t launch_near32s(const float4* pk_hi, const float4* pk_lo, const double* org, const float4* ext,
                           const double* shifts, double* partial, const NearSymLaunch& S, cudaStream_t st,
                           bool ff = false, bool refine = false);
cudaError_t launch_sym_reduce(const double* partial, int64_t n_valid, const NearSymLaunch& S, double* out_phi,
                              double* out_grad, cudaStream_t st, bool fp64 = false, bool accumulate = false);
cudaError_t launch_near64s(const double4_32a* pk, const double* shifts, double* partial, const NearSymLaunch& S,
                           cudaStream_t st);
int near64s_occupancy_ctas();
int near32s_occupancy_ctas(int img_per_g, bool ff = false, bool refine = false);
constexpr int kNear32Variants = 2;
int near64_occupancy_ctas();
// sort.cu
int sort_blocks(int64_t n);
int curve_sort_launches(int64_t n);   // kernels launch_curve_sort queues for n points
cudaError_t launch_curve_sort(const double* x, int64_t n, const double d[3], uint32_t* ka, uint32_t* va,
                               uint32_t* kb, uint32_t* vb, uint32_t* hist, cudaStream_t st);
cudaError_t launch_pack32(const double* x, const double* q, const uint32_t* perm, int64_t n, int64_t n_groups,
                          float4* pk_hi, float4* pk_lo, double* org, cudaStream_t st, double* xs = nullptr,
                          float4* ext = nullptr);
cudaError_t launch_pack64(const double* x, const double* q, int64_t n, int64_t n_pad, double4_32a* pk, cudaStream_t st);
cudaError_t launch_radix_sort(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, uint32_t* hist, int64_t n,
                              int passes, cudaStream_t st);
cudaError_t launch_pack32_groups(const double* x, const double* q, const uint32_t* perm, int64_t n_groups,
                                 const int64_t* grp_start, const int* grp_count, float4* pk_hi, float4* pk_lo,
                                 double* org, cudaStream_t st, float4* ext = nullptr);
cudaError_t launch_pack64_groups(const double* x, const double* q, int64_t n_pts, const int64_t* grp_start,
                                 const int* grp_count, double4_32a* pk, cudaStream_t st);
// far.cu
int reduce_blocks(int64_t n, int num_sms);
cudaError_t launch_validate_points(const double* y, int64_t n, const double d[3], int nblk, int* status,
                                   cudaStream_t st);
cudaError_t launch_validate(const double* x, const double* q, int64_t n, const double d[3], double* partial,
                            int nblk, int* status, cudaStream_t st);
int mean_blocks(int64_t n, int num_sms);   // grid of launch_box_mean for n charges
cudaError_t launch_box_mean(const double* x, const double* q, int64_t n, const double H[3], double* partial,
                            int nblk, cudaStream_t st);
// far field of the RBF basis (Eq. 5): phi = phi_near + C_1 + sum_t C_{t+1} / |y - x_t|, float64
cudaError_t launch_far_rbf(const double* x, int64_t n, const int* perm, const double* phi_near,
                           const double* grad_near, const double* C, const double* centres, int S, const int* status,
                           double* phi, double* grad, int* status_out, cudaStream_t st);
// trimmed near set: sum over the kept images x + p (|x + p| <= Rb) of the single box's potential
cudaError_t launch_box_mean_ball(const double* x, const double* q, const uint32_t* perm, int64_t n,
                                 const double d[3], const int K[3], double Rb, double* partial, int nblk,
                                 cudaStream_t st);
cudaError_t launch_project(const double* pinv, int rows, int M, const double* phi_check, const int* check_pos,
                           double* f, double* C, cudaStream_t st, bool layers = false);
cudaError_t launch_constant(double* C, const double* Rbox, int P, const double* mean_partial, int nblk,
                            double inv_V0, int zero_mean, cudaStream_t st);
// tab32 != nullptr: the far field in float (FP32C plans), else in double with tab64
cudaError_t launch_far_combine(const double* x, int64_t n, const int* perm, const double* phi_near,
                               const double* grad_near, const double* C, int p, double inv_R0, const double* tab64,
                               const float* tab32, const int* status, double* phi, double* grad, int* status_out,
                               cudaStream_t st);
// backward.cu
cudaError_t launch_moments(const double* x, const double* q, int64_t n, const double* C, int p, double inv_R0,
                           const double* tab, double* far_phi, double* far_grad, double* w_partial, int nblk,
                           double* w, cudaStream_t st);
int moments_blocks(int64_t n);
size_t moments_smem(int p);
cudaError_t launch_adjoint(const double* pinv, int rows, int M, const double* w, double* u, cudaStream_t st);
cudaError_t launch_check_sources32(const float4* chk_hi, const float4* chk_lo, const int* inv, int64_t n_pts, int M,
                                   const double* u, float4* out_hi, float4* out_lo, cudaStream_t st,
                                   bool layers = false);
cudaError_t launch_check_sources64(const double4_32a* chk, int64_t n_pts, int M, const double* u,
                                   double4_32a* out, cudaStream_t st);
cudaError_t launch_backward_combine(int64_t n, const int* perm, const double* q, const double* phi,
                                    const double* grad, const double* far_phi, const double* far_grad,
                                    const double* psi, const double* gpsi, const double* gE, double* dEdq,
                                    double* dEdx, cudaStream_t st);
cudaError_t launch_energy(const double* q, const double* phi, int64_t n, double* partial, int nblk, double* E,
                          cudaStream_t st);
cudaError_t set_moments_smem(size_t bytes);
}  // namespace psum

