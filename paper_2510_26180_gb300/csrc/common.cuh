// Internal declarations shared by the translation units of libklecgc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <algorithm>
#include <vector>

namespace klecgc {

constexpr int kMaxN = 128;          // largest coarse-interval count (power of 2)
constexpr int kTwiddleN = 128;      // cos/sin(2 pi t / 128) tables, t < 128

template <typename T>
struct Cplx {
    T x, y;
};

// Fine-propagator coefficients of one row i of M = I + dt (A + c I), stored
// per sample.  `l` is the LU multiplier of row i (0 for i = 0), `dinv` the
// reciprocal pivot, `wd` = dt * a_{i-1/2} / h^2 (the weight of the face left
// of row i; the off-diagonal M_{i-1,i} = M_{i,i-1} = -wd_i).
struct alignas(32) FineCoef64 {
    double l, dinv, wd, pad;
};
struct alignas(16) FineCoef32 {
    float l, dinv, wd, pad;
};


// Unevaluated sums of two floats (hi + lo, |lo| <= ulp(hi)/2): about 48-bit
// values built from FP32 operations only (Knuth's TwoSum / Dekker's
// FastTwoSum).  FP64 runs at 1/58 of the FP32 rate on this GPU, so iterates
// and accumulators of the mixed path live in this form.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = a + b;
    return make_float2(s, b - (s - a));
}
// x + y for a pair x and a float y
__device__ __forceinline__ float2 df_add(float2 x, float y) {
    float2 s = two_sum(x.x, y);
    return fast_two_sum(s.x, s.y + x.y);
}
// x - y for two pairs, rounded to one float
__device__ __forceinline__ float df_sub(float2 x, float2 y) {
    float2 s = two_sum(x.x, -y.x);
    return s.x + (s.y + (x.y - y.y));
}

// ---- the uneven batch as persistent stage kernels (k_fine32.cu, k_cgc.cu) ----
// One class of instances of equal (context, J): the device pointers and
// sizes that the stage bodies need (the arrays of one SolveRun).
struct BatchClass {
    int64_t S;                    // instances of the class
    int nx, N, K, J, R, QS;       // R, QS: rows per lane and intervals per warp of k_fine32
    int defect;                   // 1: MIXED_DEFECT (FP32 pairs), 0: MIXED
    int react, force;             // reaction / forcing terms present
    float dt_react, dt_f;         // fine step: dt c, dt f0
    double dTreact, alpha, tol;
    int kmax;
    double* U;                    // MIXED: FP64 iterate (the defect path aliases it as Udf)
    float2* Udf;
    float* fout;
    float* c32;
    double* rs;                   // MIXED: scaled CGC right-hand side
    float2* Facc0;                // MIXED_DEFECT: F accumulators (by iteration parity)
    float2* Facc1;
    Cplx<double>* p64;
    Cplx<float>* p32;
    const char* tab32;            // k_fine32 table ([S][R][32] x 24 bytes)
    const double* u0;
    const double* wT;
    const Cplx<double>* dinv64;
    const Cplx<double>* lu64;
    const Cplx<float>* dinv32;
    const Cplx<float>* lu32;
    const float* wT32;
    const double* sc64;
    const double* isc64;
    const float* sc32;
    const float* isc32;
    int* active;
    int32_t* iters;
    int32_t* status;
    unsigned long long* delta;
};
// A work item of a stage: class c, sample s of the class, and the part
// (interval group of the fine stage, x tile of the transforms, first system
// of a 128-system chunk of the shifted solves).
struct BatchTask {
    int c, part;
    int64_t s;
};
// Persistent stage kernels: grid-size CTAs pull tasks from *queue (a counter
// the caller zeroes before the launch) in list order, longest first.
// k: iteration (kdev ? *kdev : k_host).
int batch_fine_parts(int N, int R);              // fine tasks per instance
size_t batch_fine_smem(int R);
// one launch per (R, rt) group; grid <= 0: the SM count times the occupancy
void launch_batch_fine(const BatchClass* cls, const BatchTask* tasks, int ntasks, int* queue,
                       int k_host, const int* kdev, int R, int rt, int grid, cudaStream_t st);
void launch_batch_fwd(int defect, const BatchClass* cls, const BatchTask* tasks, int ntasks,
                      int* queue, int k_host, const int* kdev, int grid, cudaStream_t st);
void launch_batch_solve(int defect, const BatchClass* cls, const BatchTask* tasks, int ntasks,
                        int* queue, int grid, cudaStream_t st);
void launch_batch_inv(int defect, const BatchClass* cls, const BatchTask* tasks, int ntasks,
                      int* queue, int grid, cudaStream_t st);
// stopping rule for every instance (tasks: one per instance, part unused)
void launch_batch_conv(const BatchClass* cls, const BatchTask* inst, int64_t n, int k_host,
                       const int* kdev, int* n_active, cudaStream_t st);
int batch_transform_tile(int defect);           // x rows per transform task
int batch_grid(int kind, int defect);           // persistent grid size per stage (0 fwd, 1 solve, 2 inv)

// ---- k_field.cu ----
void launch_field(const double* xi, int64_t S, int M, const double* basis, int nf, double* a,
                  cudaStream_t st);
void launch_fine_factors(const double* a, int64_t S, int nx, double h, double dt, double react,
                         FineCoef64* f64, FineCoef32* f32, cudaStream_t st);
template <typename T>
void launch_cgc_factors(const double* a, int64_t S, int nx, double h, double dT, double react,
                        const double2* lam, int K, Cplx<T>* dinv, Cplx<T>* lu, cudaStream_t st,
                        const double* ext = nullptr);
void launch_cgc_factors32(const float* wT32, int64_t S, int nx, double dTreact,
                          const float2* lam, int K, Cplx<float>* dinv, Cplx<float>* lu,
                          cudaStream_t st);
void launch_face_weights(const double* a, int64_t S, int nf, double scale, double* w,
                         cudaStream_t st);
void launch_nonfinite_flag(const double* x, int64_t n, int* flag, cudaStream_t st);

// ---- k_guess.cu ----
template <typename T>
void launch_psi(const double* xi, int64_t S, int M, const int* degrees, int P, T* psi,
                int ld,
                cudaStream_t st);
// C[m][n] (+)= sum_k A(m,k) B(k,n); A(m,k) = A[m*lda_m + k*lda_k], B likewise,
// C row-major with leading dimension ldc; C is FP64, A/B of type T.
template <typename T>
void launch_gemm(int64_t Mr, int64_t Nc, int64_t K, const T* A, int64_t lda_m, int64_t lda_k,
                 const T* B, int64_t ldb_k, int64_t ldb_n, double* C, int64_t ldc, bool accumulate,
                 const double* row_bias, cudaStream_t st);
void launch_mean_center(double* Y, int64_t rows, int64_t cols, double* mean, cudaStream_t st);
void launch_to_float(const double* x, float* y, int64_t n, cudaStream_t st);

// ---- k_fine.cu ----
// Step 1 of Algorithm 2 plus the CGC right-hand side, internal layout
// [S][nx][N] (time fastest).  out_mode 0: r = (I + dT A) F - prev;
// out_mode 1 (defect): d = (I + dT A)(F - U_n), written as FP32.
void launch_fine_sweep_fp64(int64_t S, int N, int nx, int J, double dT, double alpha, double react,
                            double forcing, const double* U, const double* u0,
                            const FineCoef64* fc, const double* wT, double* r, const int* active,
                            cudaStream_t st, int jump = 1);
// Classical parareal correction (Algorithm 1), one thread per sample; gc: LU
// factors of I + dT(A + cI); F: fine end values; U updated in place.
void launch_parareal_correct(int64_t S, int N, int nx, double dTf, const double* u0,
                             const FineCoef64* gc, const double* F, double* U, double* scratch,
                             unsigned long long* delta, const int* active, cudaStream_t st);
// ---- k_fine32.cu ----
// FP32 increment-form fine sweep, register resident.  in_mode 0: Facc = F(start);
// in_mode 1: Facc += F0(c32 of interval n-1).  out_mode 0: r (FP64); 1: defect d32.
int fine32_rows_per_lane(int nx);
size_t fine_table32_bytes(int64_t S, int R);
void launch_fine_table32(const double* a, int64_t S, int nx, int R, double h, double dt,
                         double react, void* table, cudaStream_t st);
// in_mode 0: fout = F(start), start_n = U_{n-1} (U64, or Udf.hi), u0 for n = 0;
// in_mode 1: fout = F0(c_{n-1}), 0 for n = 0.  fout: [S][nx][N] FP32.
void launch_fine32(int64_t S, int N, int nx, int J, double dt, double react, double forcing,
                   int in_mode, const double* U64, const float2* Udf, const double* u0,
                   const float* c32, const void* table, float* fout, const int* active,
                   cudaStream_t st);
// The same with every factor in registers: W warps per pair of intervals,
// R rows per lane (32 W R >= nx + 1); the table is built from the FP64
// factors of launch_fine_factors (fine step dt).
// L >= 1 selects k_fine32r instead: one interval per warp with the factors
// in registers, L intervals per warp in turn (W unused, R rows per lane).
struct Fine32wShape {
    int W, R;
    int L = 0;
    int P = 0;   // 1: k_fine32p (halves of R rows in packed FP32x2, one interval per warp)
};
Fine32wShape fine32w_shape(int nx);
std::vector<Fine32wShape> fine32w_candidates(int nx);
bool fine32w_supported(Fine32wShape sh);
size_t fine_table32w_bytes(int64_t S, Fine32wShape sh);
void launch_fine_table32w(const FineCoef64* fc, int64_t S, int nx, Fine32wShape sh, float* table,
                          cudaStream_t st);
void launch_fine32w(Fine32wShape sh, int64_t S, int N, int nx, int J, double dt, double react,
                    double forcing, int in_mode, const double* U64, const float2* Udf,
                    const double* u0, const float* c32, const float* table, float* fout,
                    const int* active, cudaStream_t st);
size_t fine_table32r_bytes(int64_t S, int R);
void launch_fine_table32r(const FineCoef64* fc, int64_t S, int nx, int R, float* table,
                          cudaStream_t st);
bool fine32r_supported(int R, int L);
void launch_fine32r(int R, int L, int64_t S, int N, int nx, int J, double dt, double react,
                    double forcing, int in_mode, const double* U64, const float2* Udf,
                    const double* u0, const float* c32, const float* table, float* fout,
                    const int* active, cudaStream_t st);
size_t fine_table32p_bytes(int64_t S, int R);
void launch_fine_table32p(const FineCoef64* fc, int64_t S, int nx, int R, float* table,
                          cudaStream_t st);
bool fine32p_supported(int R);
void launch_fine32p(int R, int64_t S, int N, int nx, int J, double dt, double react,
                    double forcing, int in_mode, const double* U64, const float2* Udf,
                    const double* u0, const float* c32, const float* table, float* fout,
                    const int* active, cudaStream_t st);
// Any of the four: sh.P is k_fine32p; sh.L >= 1 is k_fine32r; else sh.W == 0 is k_fine32 (table of
// launch_fine_table32 with sh.R rows per lane), sh.W >= 1 is k_fine32w.
void launch_fine_any(Fine32wShape sh, int64_t S, int N, int nx, int J, double dt, double react,
                     double forcing, int in_mode, const double* U64, const float2* Udf,
                     const double* u0, const float* c32, const float* table, float* fout,
                     const int* active, cudaStream_t st);
// r = (I + dT(A + cI)) F - prev in FP64 from an FP32 F ([S][nx][N]).
void launch_jump_from_f32(int64_t S, int N, int nx, double alpha, double dTreact, const float* F,
                          const double* U, const double* wT, double* r, cudaStream_t st);
void launch_fine_sequential(int64_t S, int N, int nx, int J, double dt_forcing, const double* u0,
                            const FineCoef64* fc, double* scratch, double* U, cudaStream_t st);

// ---- k_2d.cu ---- (2D five-point problem; U/out layout [S][nx*nx][N])
// A system held by a thread-block cluster of CL CTAs (k_2d_cluster.cu).
struct ClusterPlan2D {
    int CL = 0;                  // CTAs per cluster (0: no cluster layout fits)
    int clusters = 0;            // clusters resident on the GPU at once
    size_t smem = 0;             // dynamic shared memory per CTA
    int64_t scratch_per_cta = 0; // doubles of global memory per CTA (CGC layout)
};
struct Plan2D {
    int64_t grid = 1;            // CTAs of the persistent launch
    int smem = 0;                // dynamic shared memory per CTA (0: global slices)
    int64_t per_cta = 0;         // doubles of global working storage per CTA
    int64_t scratch_doubles = 0; // total global working storage
    ClusterPlan2D cl;            // kind 2: the cluster layout, when cl.CL > 0
};
// kind 0: fine propagator, 1: shifted CGC solves, 2: mixed fine, 3: mixed CGC,
// 4 / 5: fine / CGC with advection (BiCGStab); items = work items.  Kind 2
// takes the cluster layout when one system does not fit one CTA's shared
// memory, or always with force_cluster; kind 3 (the mixed CGC) likewise,
// with its FP64 residual in scratch_doubles of global memory.
Plan2D plan_2d(int kind, int nx, int64_t items, bool force_cluster = false);
ClusterPlan2D fine2d_cluster_plan(int nx);
ClusterPlan2D cgc2d_cluster_plan(int nx);
void launch_cgc_solve2d_mixed_cl(const ClusterPlan2D& p, int64_t S, int K, int nx, double dTc,
                                 const double2* lam, const double* wdT, double rtol, double tin,
                                 int maxit, Cplx<double>* pio, const int* active, int* ifail,
                                 unsigned long long* itcount, double* scratch, int64_t grid,
                                 cudaStream_t st);
void launch_fine2d_mixed_cl(const ClusterPlan2D& p, int64_t S, int N, int nx, int J, double dtc,
                            double dtf, double alpha, int mode, const double* U, const double* u0,
                            const double* wdt, double rtol, double tin, int maxit, double* out,
                            const int* active, int* ifail, unsigned long long* itcount,
                            cudaStream_t st);
// mode 0: r = (I + L_dT) F(start) - prev per (s, n); mode 1: sequential fine
// solution out[s][.][n] per s.  wdt: [S][2 nx (nx+1)] weights dt a / h^2.
// adv = dt b0 of the upwind convection (advection-diffusion, BiCGStab, plan
// kind 4), 0 for the symmetric problem (CG, plan kind 0).
void launch_fine2d(const Plan2D& pl, int64_t S, int N, int nx, int J, double dtc, double dtf,
                   double adv, double alpha, int mode, const double* U, const double* u0,
                   const double* wdt, double rtol, int maxit, double* out, const int* active,
                   int* ifail, unsigned long long* itcount, double* scratch, cudaStream_t st);
// The same with each backward-Euler step solved by FP64 iterative refinement
// around an FP32 Jacobi-PCG (inner relative tolerance tin, plan kind 2).
void launch_fine2d_mixed(const Plan2D& pl, int64_t S, int N, int nx, int J, double dtc,
                         double dtf, double alpha, int mode, const double* U, const double* u0,
                         const double* wdt, double rtol, double tin, int maxit, double* out,
                         const int* active, int* ifail, unsigned long long* itcount,
                         double* scratch, cudaStream_t st);
// (lambda_k I + L_dT) q = p in place by FP64 refinement around FP32 COCG (plan kind 3).
void launch_cgc_solve2d_mixed(const Plan2D& pl, int64_t S, int K, int nx, double dTc,
                              const double2* lam, const double* wdT, double rtol, double tin,
                              int maxit, Cplx<double>* p, const int* active, int* ifail,
                              unsigned long long* itcount, double* scratch, cudaStream_t st);
// (lambda_k I + L_dT) q = p in place, p: [S][nx*nx][K]; wdT = dT a / h^2;
// adv = dT b0 (BiCGStab, plan kind 5) or 0 (COCG, plan kind 1).
void launch_cgc_solve2d(const Plan2D& pl, int64_t S, int K, int nx, double dTc, double adv,
                        const double2* lam, const double* wdT, double rtol, int maxit,
                        Cplx<double>* p, const int* active, int* ifail,
                        unsigned long long* itcount, double* scratch, cudaStream_t st);

// ---- k_batch.cu ---- (uneven batch)
void launch_gather_rows(const double* in, const int64_t* idx, int64_t S, int M, double* out,
                        cudaStream_t st);
void launch_scatter_blocks(const double* src, const int64_t* off, int64_t S, int64_t block,
                           double* dst, cudaStream_t st);

// ---- k_tc.cu ---- (tcgen05 surrogate guess)
// K extent of the padded psi / W^T rows (multiple of the MMA chunk).
int guess_tc_k_padded(int P);
// Wt[c][j] = W[j][c] (j < P), zero up to Kp.
void launch_pad_transpose(const float* W, int P, int64_t NC, int Kp, float* Wt, cudaStream_t st);
// hi = TF32 rounding of x, lo = x - hi.
void launch_split_tf32(const float* x, int64_t n, float* hi, float* lo, cudaStream_t st);
// U[s][c] = ubar[c] + sum_j psi[s][j] Wt[c][j] with psi and Wt split into TF32
// head and tail ([S][Kp], [NC][Kp], zero-padded, 16-byte aligned; NC even),
// loaded by TMA; *err = 1 if a pipeline wait ran out of its budget.  With
// ubar_df (ubar as FP32 pairs) non-null, each U value is stored as the FP32
// pair (hi, lo) in its 8 bytes.  Returns an error if the tensor maps cannot
// be encoded.
cudaError_t launch_guess_tc(int64_t S, int64_t NC, int Kp, const float* psi_hi,
                            const float* psi_lo, const float* Wt_hi, const float* Wt_lo,
                            const double* ubar, const float2* ubar_df, double* U, int* err,
                            cudaStream_t st);

// ---- k_nonlinear.cu ---- (kind 1 cubic reaction, kind 2 Burgers-type
// convection; simplified-Newton CGC; wf = a / h^2; c the problem's coefficient)
// F by Newton backward-Euler steps and, with jump, b = F - G(prev) per (s, n)
// (else F); scratch: 4 S nx N doubles.
void launch_fine_newton(int kind, int64_t S, int N, int nx, int J, double dT, double alpha,
                        double c, double f0, int jump, const double* U, const double* u0,
                        const double* wf, double* b, double* scratch, const int* active,
                        int* ifail, unsigned long long* itcount, cudaStream_t st);
// N J sequential Newton steps of dt per sample (one thread each); scratch 4 nx S.
void launch_sequential_newton(int kind, int64_t S, int N, int nx, int J, double dt, double c,
                              double f0, const double* u0, const double* wf, double* scratch,
                              double* U, int* ifail, cudaStream_t st);
// Kind 2: face couplings lo, up ([S][nx+1], dT-scaled) of the averaged
// Jacobian and the right-hand side of eq. Newton2.
void launch_nl_prep_burgers(int64_t S, int N, int nx, double dT, double c, double f0,
                            const double* u, const double* b, const double* wf, double* rhs,
                            double* lo, double* up, const int* active, cudaStream_t st);
// Factors of lambda_k I + dT K from the face couplings (k_cgc_solve layout).
void launch_cgc_factors_faces(int64_t S, int nx, const double* lo, const double* up,
                              const double2* lam, int K, Cplx<double>* dinv, Cplx<double>* lu,
                              const int* active, cudaStream_t st);
// Classical parareal correction with Newton G; scratch 5 nx S doubles.
void launch_parareal_correct_newton(int kind, int64_t S, int N, int nx, double dT, double c,
                                    double f0, const double* u0, const double* wf,
                                    const double* F, double* U, double* scratch,
                                    unsigned long long* delta, const int* active, int* ifail,
                                    cudaStream_t st);
// e = c (3 mean_n (u - b)^2 - 1) per row and the right-hand side of eq. Newton2.
void launch_nl_prep(int64_t S, int N, int nx, double dT, double c, double f0, const double* u,
                    const double* b, const double* wf, double* rhs, double* e, const int* active,
                    cudaStream_t st);

// ---- k_band.cu ---- (2D banded LU, small grids)
// Doubles (complex values for the CGC) of one band matrix: nx^2 (2 nx + 1).
int64_t band_doubles(int nx);
// Factors of I + step (A + cI) + convection per sample; w: step a / h^2
// faces [S][2 nx (nx+1)], dtc = step c, adv = step b0; Bf: [S][band].
void launch_band_factor_fine(int64_t S, int nx, const double* wdt, double dtc, double adv_dt,
                             double* Bf, cudaStream_t st);
// Factors of lambda_k I + dT (A + cI) + convection per (s, k); Bc: [S][K][band].
void launch_band_factor_cgc(int64_t S, int K, int nx, const double* wdT, double dTc,
                            double adv_dT, const double2* lam, double2* Bc, cudaStream_t st);
// F by banded solves, modes and outputs as launch_fine2d; x: scratch
// [S][nx^2][N] (mode 0) or [nx^2][S] (mode 1).
void launch_band_fine(int64_t S, int N, int nx, int J, double dtc, double dtf, double adv_dt,
                      double alpha, int mode, const double* U, const double* u0,
                      const double* wdt, const double* Bf, double* x, double* out,
                      const int* active, cudaStream_t st);
// (lambda_k I + L_dT) q = p in place, p: [S][nx^2][K].
void launch_band_cgc(int64_t S, int K, int nx, const double2* Bc, Cplx<double>* p,
                     const int* active, cudaStream_t st);

// ---- k_offline.cu ---- (Algorithm 3 steps 2-5 on the device)
// Eigenpairs of the symmetric n x n A (overwritten; its diagonal ends as the
// eigenvalues) by parallel cyclic threshold Jacobi, eigenvectors as the rows
// of Vt; cooperative launch; rot: (n+1)/2 double2, part: 2 nparts doubles;
// *info = sweeps taken, or -1 when max_sweeps left an off-diagonal entry
// above tol ||A||_F.
cudaError_t launch_jacobi_eig(int n, double* A, double* Vt, double2* rot, double* part, int nparts,
                              double tol, int max_sweeps, int* info, cudaStream_t st);
void launch_transpose64(const double* in, int rows, int cols, double* out, cudaStream_t st);
// Es[k][j] = Vt[idx_k][j] / sqrt(ev_k nt), Dc[k][j] = sqrt(nt) Vt[idx_k][j].
void launch_gather_modes(const double* Vt, int nt, const int* idx, const double* ev, int MQ,
                         double* Es, double* Dc, cudaStream_t st);
// X = argmin ||B X - D|| (Householder QR, one CTA), Bc [n][m] and Dc [r][m]
// column-contiguous (overwritten), X [n][r] scaled by colscale per column;
// v: m doubles; *info = 1 when rank deficient.
void launch_lstsq_qr(int m, int n, int r, double* Bc, double* Dc, double* v,
                     const double* colscale, double* X, int* info, cudaStream_t st);

// ---- k_cgc.cu ----
// Step (a): p[s][i][k] = sum_j alpha^{j/N} r[s][i][j] exp(-2 pi i j k / N), k <= N/2.
template <typename T, typename TIN>
void launch_cgc_forward(int64_t S, int N, int nx, const TIN* r, const T* scale, Cplx<T>* p,
                        const int* active, cudaStream_t st);
// Step (b): (lambda_k I + dT A) q_k = p_k in place.
template <typename T, typename TW>
void launch_cgc_solve(int64_t S, int K, int nx, const Cplx<T>* dinv, const Cplx<T>* lu,
                      const TW* wT, Cplx<T>* p, const int* active, cudaStream_t st);
// Step (a) with the FP32 fine result folded in (defect path).  Facc_out =
// Facc_in + fout (Facc_in null on the first iteration); then
// d = (I + dT(A+cI)) (Facc_out - U) on pairs U, Facc (FP32 ops only).
// Iteration k (kdev ? *kdev : k) reads F(U^{k-1}) from Facc[(k-1) & 1] (none at
// k = 0) and writes F(U^k) to Facc[k & 1].
void launch_cgc_forward_df(int64_t S, int N, int nx, const float* fout, float2* Facc0,
                           float2* Facc1, int k, const int* kdev, const float2* Udf,
                           const double* wT, double dTreact, const float* scale, Cplx<float>* p,
                           const int* active, cudaStream_t st);
// Step (a) for the mixed path: the CGC right-hand side accumulated in FP64,
// pre-scaled (rs = alpha^{n/N} r): formed in FP64 from F(start) = fout when
// c32 is NULL (first iteration), else incremented by the FP32 flux-form
// (I + dT(A + cI)) F0(c_{n-1}) - c_{n-1}; then p = 2 DFT_n(rs).
void launch_cgc_forward_acc(int64_t S, int N, int nx, const float* fout, const float* c32,
                            const double* U, const double* wT, double dTreact, double alpha,
                            const double* scale, const float* scale32, double* rs,
                            Cplx<double>* p, const int* active, cudaStream_t st);
// Step (c) + pair update (defect path): Udf += u, c32 = u, delta = max|u|.
void launch_cgc_inverse_df(int64_t S, int N, int nx, const Cplx<float>* q, const float* iscale,
                           float2* Udf, unsigned long long* delta, float* c32, const int* active,
                           cudaStream_t st);
// FP64 [S][nx][N] <-> pairs, in place (same 8 bytes per value).
void launch_to_pairs(double* U, int64_t n, cudaStream_t st);
// pairs [S][nx][N] -> FP64 [S][N][nx]
void launch_pairs_transpose_out(const float2* in, double* out, int64_t S, int nx, int N,
                                cudaStream_t st);
// Step (c) + update: u_j = alpha^{-j/N} (1/N) sum_k q_k exp(+2 pi i j k / N).
// mode 0: U <- u, delta = max|u - U_old|;  mode 1: U <- U + u, delta = max|u|;
// mode 2: out <- u (no delta).  In modes 0 and 1 the increment U_new - U_old is
// also stored as FP32 in c32 when c32 is not null.
template <typename T>
void launch_cgc_inverse(int64_t S, int N, int nx, const Cplx<T>* q, const T* iscale, double* U,
                        int mode, unsigned long long* delta, float* c32, const int* active,
                        cudaStream_t st);
void launch_convergence(int64_t S, int iter, int kmax, double tol, unsigned long long* delta,
                        int* active, int32_t* iters, int32_t* status, int* n_active,
                        cudaStream_t st, const int* kdev = nullptr);
// Device-driven loop: the tail of a WHILE-node body (k += 1; continue while
// any sample is active and k < kmax) and a one-value setter.
void launch_loop_tail(int* kdev, const int* n_active, int kmax, cudaGraphConditionalHandle h,
                      cudaStream_t st);
void launch_set_int(int* p, int v, cudaStream_t st);
// [S][A][B] -> [S][B][A] (FP64).
void launch_transpose(const double* in, double* out, int64_t S, int A, int B, cudaStream_t st);

// ---- k_mlp.cu ----
}  // namespace klecgc
#include <cuda_bf16.h>
namespace klecgc {
void launch_gemm_bf16(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16* A, int lda,
                      const __nv_bfloat16* B, int ldb, const float* bias, const float* zmask,
                      int ldz, float* C, int ldc, __nv_bfloat16* Cb, int ldcb, bool relu,
                      cudaStream_t st);
// C = A B^T on the tcgen05 tensor cores (BF16 K-major operands [M][K], [N][K],
// FP32 accumulation in tensor memory), same epilogue as launch_gemm_bf16;
// err: the bounded-wait flag (set on a timeout).  gemm_bf16_tc_ok: the sizes
// and alignments TMA needs.
bool gemm_bf16_tc_ok(int M, int N, int K, const void* A, int lda, const void* B, int ldb);
cudaError_t launch_gemm_bf16_tc(int M, int N, int K, const __nv_bfloat16* A, int lda,
                                const __nv_bfloat16* B, int ldb, const float* bias,
                                const float* zmask, int ldz, float* C, int ldc,
                                __nv_bfloat16* Cb, int ldcb, bool relu, int* err,
                                cudaStream_t st);
void launch_transpose_bf16(const __nv_bfloat16* in, int R, int Cc, int ld_in, __nv_bfloat16* out,
                           cudaStream_t st);
void launch_mlp_gather(int B, int M, int D, const int* perm, int b0, const double* xi,
                       const float* targ, const float* mean, const float* inv_std,
                       __nv_bfloat16* X, float* T, cudaStream_t st);
void launch_mse(int64_t n, float gscale, float lscale, const float* Y, const float* T, float* dY,
                __nv_bfloat16* dYb, float* loss, cudaStream_t st);
void launch_colsum(int B, int D, const float* dZ, float* db, cudaStream_t st);
void launch_adam(int64_t n, float lr, int t, float* th, const float* g, float* m, float* v,
                 __nv_bfloat16* thb, cudaStream_t st);
void launch_f32_to_bf16(int64_t n, const float* x, __nv_bfloat16* y, cudaStream_t st);
void launch_downsample(int64_t rows, int nx, const double* U, float* T, cudaStream_t st);
void launch_upsample(int64_t S, int N, int nx, const float* Y, const float* mean,
                     const float* stdv, double* U, bool accumulate, cudaStream_t st);
// a -= b elementwise (FP32).
void launch_sub_f32(int64_t n, float* a, const float* b, cudaStream_t st);
void launch_colstats(int64_t n, int D, const float* T, float* mean, float* stdv, float* inv_std,
                     cudaStream_t st);
void launch_nonfinite_f32(int64_t n, const float* x, int* flag, cudaStream_t st);

// Thread-local last-error detail.
void set_error(const std::string& msg);

// Read-only view of a context's problem data (defined in api.cu).
struct CtxView {
    const double* basis;  // [M][nx+1] field basis at the faces
    const double* u0;     // [nx]
    int nx, M, device;
    double h, T, reaction, forcing;
    int dim;
    int reaction_kind;
};
}  // namespace klecgc
struct klecgc_ctx;
namespace klecgc {
bool ctx_view(const klecgc_ctx* ctx, CtxView* out);

}  // namespace klecgc

#define KLECGC_CUDA_TRY(expr)                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            klecgc::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));              \
            return e_ == cudaErrorMemoryAllocation ? KLECGC_E_OUT_OF_MEMORY : KLECGC_E_CUDA;   \
        }                                                                                      \
    } while (0)
