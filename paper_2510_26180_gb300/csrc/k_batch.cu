// Gather/scatter of the uneven batch (klecgc_solve_batch): instances are
// grouped into classes of equal (context, J); a class's inputs are gathered
// into a contiguous block and its results scattered back to the packed
// per-instance output.
#include "common.cuh"

namespace klecgc {

// out[s][m] = in[idx[s]][m]
__global__ void k_gather_rows(const double* __restrict__ in, const int64_t* __restrict__ idx,
                              int64_t S, int M, double* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * M) return;
    const int64_t s = t / M;
    const int m = (int)(t - s * M);
    out[t] = in[idx[s] * M + m];
}

void launch_gather_rows(const double* in, const int64_t* idx, int64_t S, int M, double* out,
                        cudaStream_t st) {
    const int64_t n = S * M;
    if (n == 0) return;
    k_gather_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, idx, S, M, out);
}

// dst[off[s] + e] = src[s * block + e], e < block; grid.y covers the block.
__global__ void k_scatter_blocks(const double* __restrict__ src, const int64_t* __restrict__ off,
                                 int64_t block, double* __restrict__ dst) {
    const int64_t s = blockIdx.x;
    const double* a = src + s * block;
    double* b = dst + off[s];
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < block;
         e += (int64_t)gridDim.y * blockDim.x)
        b[e] = a[e];
}

void launch_scatter_blocks(const double* src, const int64_t* off, int64_t S, int64_t block,
                           double* dst, cudaStream_t st) {
    if (S == 0 || block == 0) return;
    int64_t gy = (block + 255) / 256;
    if (gy > 64) gy = 64;
    k_scatter_blocks<<<dim3((unsigned)S, (unsigned)gy), 256, 0, st>>>(src, off, block, dst);
}

}  // namespace klecgc
