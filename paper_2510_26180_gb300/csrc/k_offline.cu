// Offline stage of Algorithm 3 on the device (steps 2-5): the eigenpairs of
// the snapshot Gram matrix (method of snapshots, eq. of the snapshot KL) and
// the least-squares fit of the gPC coefficients (eq. of the LS problem).
//
// Eigenpairs: parallel cyclic Jacobi.  A symmetric n x n matrix is reduced
// by sweeps of plane rotations; each sweep runs m - 1 steps (m = n rounded up
// to even), and a step rotates the m/2 disjoint index pairs of a round-robin
// schedule at once: A <- J^T A J with J the product of the step's rotations
// (each chosen to annihilate its pair's off-diagonal entry, Golub-Van Loan
// Algorithm 8.5.2), accumulated into V^T <- J^T V^T.  The phases of a step
// (angles; rows; columns) are separated by grid-wide barriers of a
// cooperative launch.  Threshold variant: with tau = tol ||A||_F, a pair
// whose entry is at most tau is not rotated, and the sweeps stop when no
// off-diagonal entry exceeds tau (the eigenvalues are then within n tau of
// those of A).  This leaves alone the rounding-level entries of the large
// cluster of near-zero eigenvalues of a rank-deficient Gram matrix, which a
// test on the total off-diagonal mass would keep rotating for many sweeps.
// A sweep that reduces the mass above tau less than 4x once it is below
// 1e-20 ||A||_F^2 also ends the iteration (rounding floor).  The diagonal then
// holds the eigenvalues and the rows of V^T the eigenvectors.
//
// Least squares: Householder QR of the design matrix (one CTA, columns
// stored contiguously), applied to the right-hand sides, then back
// substitution.
#include <cooperative_groups.h>

#include "common.cuh"

namespace klecgc {

namespace cg = cooperative_groups;

namespace {

constexpr int kJacobiThreads = 256;
constexpr int kQrThreads = 1024;

// Pair k of step t of the round-robin schedule over m (even) indices: index
// 0 stays, the others rotate by t positions; returns p < q.
__device__ __forceinline__ void rr_pair(int m, int t, int k, int& p, int& q) {
    const int a = k == 0 ? 0 : 1 + (k - 1 + t) % (m - 1);
    const int b = 1 + (m - 2 - k + t) % (m - 1);   // position m-1-k (never 0)
    p = a < b ? a : b;
    q = a < b ? b : a;
}

__device__ __forceinline__ double block_sum_1(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    return s;
}

__global__ void __launch_bounds__(kJacobiThreads) k_jacobi_eig(
    int n, double* __restrict__ A, double* __restrict__ Vt, double2* __restrict__ rot,
    double* __restrict__ part, double tol2, int max_sweeps, int* __restrict__ info) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double red[32];
    const int m = n + (n & 1), half = m / 2;
    const int64_t nn = (int64_t)n * n;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = tid; e < nn; e += nth) Vt[e] = (e / n == e % n) ? 1.0 : 0.0;
    // ||A||_F^2 (every block sums the partials in the same order, so all
    // decisions below are uniform across the grid)
    double tot = 0.0;
    for (int64_t e = tid; e < nn; e += nth) tot = fma(A[e], A[e], tot);
    tot = block_sum_1(tot, red);
    if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = tot;
    grid.sync();
    double st = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) st += part[2 * b + 1];
    const double tau2 = tol2 * st;   // tau^2
    const double tau = sqrt(tau2);
    int sweep = 0;
    bool converged = false;
    double prev = 0.0;   // off-diagonal mass above tau after the previous sweep
    for (;;) {
        double off = 0.0;
        for (int64_t e = tid; e < nn; e += nth) {
            const double a = A[e];
            if (e / n != e % n && a * a > tau2) off = fma(a, a, off);
        }
        off = block_sum_1(off, red);
        if (threadIdx.x == 0) part[2 * blockIdx.x] = off;
        grid.sync();
        double so = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) so += part[2 * b];
        if (so == 0.0 || (sweep > 0 && so <= 1e-20 * st && so > 0.25 * prev)) {
            converged = true;
            break;
        }
        prev = so;
        if (sweep == max_sweeps) break;
        ++sweep;
        for (int t = 0; t < m - 1; ++t) {
            // angles
            for (int64_t k = tid; k < half; k += nth) {
                int p, q;
                rr_pair(m, t, (int)k, p, q);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = A[(int64_t)p * n + q];
                    if (fabs(apq) > tau) {
                        const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                    }
                }
                rot[k] = make_double2(c, s);
            }
            grid.sync();
            // rows p, q of A and of V^T: J^T applied from the left
            for (int64_t e = tid; e < (int64_t)half * n; e += nth) {
                const int k = (int)(e / n), j = (int)(e - (int64_t)k * n);
                const double2 cs = rot[k];
                if (cs.y == 0.0) continue;
                int p, q;
                rr_pair(m, t, k, p, q);
                const double ap = A[(int64_t)p * n + j], aq = A[(int64_t)q * n + j];
                A[(int64_t)p * n + j] = cs.x * ap - cs.y * aq;
                A[(int64_t)q * n + j] = cs.y * ap + cs.x * aq;
                const double vp = Vt[(int64_t)p * n + j], vq = Vt[(int64_t)q * n + j];
                Vt[(int64_t)p * n + j] = cs.x * vp - cs.y * vq;
                Vt[(int64_t)q * n + j] = cs.y * vp + cs.x * vq;
            }
            grid.sync();
            // columns p, q of A: J from the right
            for (int64_t e = tid; e < (int64_t)half * n; e += nth) {
                const int k = (int)(e / n), i = (int)(e - (int64_t)k * n);
                const double2 cs = rot[k];
                if (cs.y == 0.0) continue;
                int p, q;
                rr_pair(m, t, k, p, q);
                const double ap = A[(int64_t)i * n + p], aq = A[(int64_t)i * n + q];
                A[(int64_t)i * n + p] = cs.x * ap - cs.y * aq;
                A[(int64_t)i * n + q] = cs.y * ap + cs.x * aq;
            }
            grid.sync();
        }
    }
    if (tid == 0) *info = converged ? sweep : -1;
}

// out[j][i] = in[i][j] (FP64; in is rows x cols).
__global__ void k_transpose64(const double* __restrict__ in, int rows, int cols,
                              double* __restrict__ out) {
    __shared__ double tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        tile[dy][threadIdx.x] = (r < rows && c < cols) ? in[(int64_t)r * cols + c] : 0.0;
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int c = c0 + dy, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(int64_t)c * rows + r] = tile[threadIdx.x][dy];
    }
}

// Kept modes, from the eigenvector rows of V^T (idx: the MQ largest
// eigenvalues ev in descending order):
//   Es[k][j] = V^T[idx_k][j] / sqrt(ev_k n_t)   (g_k = sum_j Es[k][j] ytilde_j)
//   Dc[k][j] = sqrt(n_t) V^T[idx_k][j]          (zeta_k(xi_j), column k of D)
__global__ void k_gather_modes(const double* __restrict__ Vt, int nt, const int* __restrict__ idx,
                               const double* __restrict__ ev, int MQ, double* __restrict__ Es,
                               double* __restrict__ Dc) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)MQ * nt) return;
    const int k = (int)(e / nt), j = (int)(e - (int64_t)k * nt);
    const double v = Vt[(int64_t)idx[k] * nt + j];
    Es[e] = v / sqrt(ev[k] * nt);
    Dc[e] = sqrt((double)nt) * v;
}

// min ||B X - D|| for every column of D: Bc [n][m] (column j contiguous),
// Dc [r][m]; one CTA.  X [n][r] row-major, scaled by colscale[k] per column
// k.  *info = 0, or 1 when R has a zero on its diagonal (rank deficient).
__global__ void __launch_bounds__(kQrThreads) k_lstsq_qr(int m, int n, int r,
                                                         double* __restrict__ Bc,
                                                         double* __restrict__ Dc,
                                                         double* __restrict__ v,
                                                         const double* __restrict__ colscale,
                                                         double* __restrict__ X,
                                                         int* __restrict__ info) {
    __shared__ double red[32];
    __shared__ int bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) bad = 0;
    for (int k = 0; k < n; ++k) {
        double* bk = Bc + (int64_t)k * m;
        double s2 = 0.0;
        for (int i = k + threadIdx.x; i < m; i += blockDim.x) s2 = fma(bk[i], bk[i], s2);
        const double nrm = sqrt(block_sum_1(s2, red));
        if (nrm == 0.0) {
            if (threadIdx.x == 0) bad = 1;
            break;   // uniform
        }
        const double alpha = bk[k] > 0.0 ? -nrm : nrm;
        double vn = 0.0;
        for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
            const double vi = bk[i] - (i == k ? alpha : 0.0);
            v[i] = vi;
            vn = fma(vi, vi, vn);
        }
        vn = block_sum_1(vn, red);   // its barrier also publishes v
        if (vn == 0.0) continue;     // uniform
        const double sc = 2.0 / vn;
        // H = I - 2 v v^T / (v^T v) on columns k..n-1 of B and on D, a warp per column
        for (int c = warp; c < (n - k) + r; c += nw) {
            double* col = c < n - k ? Bc + (int64_t)(k + c) * m : Dc + (int64_t)(c - (n - k)) * m;
            double s = 0.0;
            for (int i = k + lane; i < m; i += 32) s = fma(v[i], col[i], s);
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            s *= sc;
            for (int i = k + lane; i < m; i += 32) col[i] = fma(-s, v[i], col[i]);
        }
        __syncthreads();
    }
    __syncthreads();
    if (!bad) {
        // R X = (Q^T D)[0:n], one thread per column of D
        for (int j = threadIdx.x; j < r; j += blockDim.x) {
            const double* dj = Dc + (int64_t)j * m;
            for (int i = n - 1; i >= 0; --i) {
                double s = dj[i];
                for (int t = i + 1; t < n; ++t) s = fma(-Bc[(int64_t)t * m + i], X[(int64_t)t * r + j], s);
                const double rii = Bc[(int64_t)i * m + i];
                if (rii == 0.0) {
                    bad = 1;   // benign race: every writer stores 1
                    break;
                }
                X[(int64_t)i * r + j] = s / rii;
            }
        }
        __syncthreads();
        if (!bad)
            for (int64_t e = threadIdx.x; e < (int64_t)n * r; e += blockDim.x)
                X[e] *= colscale[e % r];
    }
    if (threadIdx.x == 0) *info = bad;
}

}  // namespace

cudaError_t launch_jacobi_eig(int n, double* A, double* Vt, double2* rot, double* part, int nparts,
                              double tol, int max_sweeps, int* info, cudaStream_t st) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jacobi_eig, kJacobiThreads, 0);
    const int64_t m = n + (n & 1);
    const int64_t need = (m / 2 * (int64_t)n + kJacobiThreads - 1) / kJacobiThreads;
    int blocks = sms * (occ > 0 ? occ : 1);
    if (blocks > nparts) blocks = nparts;
    if (blocks > need) blocks = (int)need;
    if (blocks < 1) blocks = 1;
    double tol2 = tol * tol;
    void* args[] = {&n, &A, &Vt, &rot, &part, &tol2, &max_sweeps, &info};
    return cudaLaunchCooperativeKernel((const void*)k_jacobi_eig, dim3(blocks),
                                       dim3(kJacobiThreads), args, 0, st);
}

void launch_transpose64(const double* in, int rows, int cols, double* out, cudaStream_t st) {
    if (rows == 0 || cols == 0) return;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    k_transpose64<<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, out);
}

void launch_gather_modes(const double* Vt, int nt, const int* idx, const double* ev, int MQ,
                         double* Es, double* Dc, cudaStream_t st) {
    const int64_t tot = (int64_t)MQ * nt;
    if (tot == 0) return;
    k_gather_modes<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Vt, nt, idx, ev, MQ, Es, Dc);
}

void launch_lstsq_qr(int m, int n, int r, double* Bc, double* Dc, double* v,
                     const double* colscale, double* X, int* info, cudaStream_t st) {
    k_lstsq_qr<<<1, kQrThreads, 0, st>>>(m, n, r, Bc, Dc, v, colscale, X, info);
}

}  // namespace klecgc
