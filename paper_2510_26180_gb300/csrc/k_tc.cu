// Surrogate guess on the fifth-generation tensor cores (hot-path row a2,
// Algorithm 3 step 6):  U[s][c] = ubar[c] + sum_j psi[s][j] W[j][c].
//
// One CTA computes a 128 x 256 output tile with tcgen05.mma (kind::tf32, FP32
// accumulation in tensor memory).  To keep FP32 accuracy each operand is
// split into a TF32 head and an FP32 tail, x = hi + lo, and the tile
// accumulates hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding).
// The 128 threads stage K-chunks of 32 of psi (A, 128 x 32) and W^T (B,
// 256 x 32) into shared memory in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices), double-buffered: while the tensor core
// multiplies one stage the threads fill the other.  One thread issues the
// MMAs and commits them to the stage's mbarrier; every wait on an mbarrier is
// bounded by a clock budget, after which the CTA sets the error flag, and
// the CTA frees its tensor memory before it returns.
//
// Shared-memory layout of one operand chunk (rows R, 32 K values): core
// matrix (r / 8, k / 4) at byte (r/8 * 8 + k/4) * 128, row r % 8 at +16 (r % 8),
// so the descriptor's leading byte offset (between core matrices along K) is
// 128 and the stride byte offset (between 8-row groups) is 1024.  (Either
// reading of the two offsets addresses only the operand's own chunk.)
#include <cstdint>

#include "common.cuh"

namespace klecgc {

namespace {

constexpr int TM = 128, TN = 256, TK = 32;
constexpr int A_BYTES = TM * TK * 4, B_BYTES = TN * TK * 4;   // one split half
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;          // hi and lo of A and B
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 64;
constexpr long long kWaitCycles = 200000000LL;                   // ~0.1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Loads 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Stages rows [r0, r0 + rows) of a K-major FP32 matrix (leading dimension ld,
// row limit nrows, K columns k0 .. k0+31) as TF32 head and tail.  Thread t
// handles rows t, t + 128, ...: a warp writes 32 consecutive 16-byte core
// rows (conflict-free).
template <int ROWS>
__device__ __forceinline__ void stage_split(const float* __restrict__ g, int64_t ld,
                                            int64_t r0, int64_t nrows, int k0, char* hi,
                                            char* lo) {
#pragma unroll
    for (int rr = 0; rr < ROWS / 128; ++rr) {
        const int r = threadIdx.x + rr * 128;
        const int64_t gr = r0 + r;
        float4 x[8];
#pragma unroll
        for (int kq = 0; kq < 8; ++kq)
            x[kq] = gr < nrows ? *reinterpret_cast<const float4*>(g + gr * ld + k0 + 4 * kq)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int kq = 0; kq < 8; ++kq) {
            const int off = ((r >> 3) * 8 + kq) * 128 + (r & 7) * 16;
            float4 h, l;
            h.x = tf32_hi(x[kq].x);
            h.y = tf32_hi(x[kq].y);
            h.z = tf32_hi(x[kq].z);
            h.w = tf32_hi(x[kq].w);
            l.x = x[kq].x - h.x;
            l.y = x[kq].y - h.y;
            l.z = x[kq].z - h.z;
            l.w = x[kq].w - h.w;
            *reinterpret_cast<float4*>(hi + off) = h;
            *reinterpret_cast<float4*>(lo + off) = l;
        }
    }
}

__global__ void __launch_bounds__(128, 1) k_guess_tc(int64_t S, int64_t NC, int Kp,
                                                    const float* __restrict__ psi,
                                                    const float* __restrict__ Wt,
                                                    const double* __restrict__ ubar,
                                                    double* __restrict__ U, int* __restrict__ err) {
    extern __shared__ __align__(1024) char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE_BYTES);  // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
    // once a CTA has timed out the launch's result is void: later CTAs skip
    if (*reinterpret_cast<volatile int*>(err)) return;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = make_idesc(TM, TN);
    bool ok = true;

    const int nch = Kp / TK;
    for (int c = 0; c < nch; ++c) {
        const int st = c & 1;
        char* base = smem + st * STAGE_BYTES;
        char* Ahi = base;
        char* Alo = base + A_BYTES;
        char* Bhi = base + 2 * A_BYTES;
        char* Blo = Bhi + B_BYTES;
        // the MMAs that last read this stage (chunk c - 2) must have finished
        if (c >= 2 && ok) ok = mbar_wait(&bar[st], ((c - 2) >> 1) & 1);
        stage_split<TM>(psi, Kp, m0, S, c * TK, Ahi, Alo);
        stage_split<TN>(Wt, Kp, n0, NC, c * TK, Bhi, Blo);
        // generic-proxy writes -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TK / 8; ++kk) {
                // K step of 8 TF32 values = 2 core matrices along K
                const uint32_t ko = kk * 2 * 128;
                const uint64_t ah = make_desc(smem_u32(Ahi) + ko, 128, 1024);
                const uint64_t al = make_desc(smem_u32(Alo) + ko, 128, 1024);
                const uint64_t bh = make_desc(smem_u32(Bhi) + ko, 128, 1024);
                const uint64_t bl = make_desc(smem_u32(Blo) + ko, 128, 1024);
                mma_tf32(tmem, ah, bh, idesc, (c | kk) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, idesc, 1u);
                mma_tf32(tmem, al, bh, idesc, 1u);
            }
            mma_commit(&bar[st]);
        }
    }
    // all MMAs done: the last commit of each stage
    if (ok && nch >= 2) ok = mbar_wait(&bar[(nch - 2) & 1], ((nch - 2) >> 1) & 1);
    if (ok && nch >= 1) ok = mbar_wait(&bar[(nch - 1) & 1], ((nch - 1) >> 1) & 1);
    ok = __syncthreads_and(ok);   // uniform: the epilogue's TMEM loads are warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (ok) {
        // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int cb = 0; cb < TN; cb += 32) {
            float v[32];
            tmem_ld32(lane_addr + cb, v);
            if (row < S) {
                double* out = U + row * NC + n0 + cb;
                if (n0 + cb + 32 <= NC) {
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const double2 b = *reinterpret_cast<const double2*>(ubar + n0 + cb + i);
                        *reinterpret_cast<double2*>(out + i) =
                            make_double2(b.x + (double)v[i], b.y + (double)v[i + 1]);
                    }
                } else {
                    for (int i = 0; i < 32 && n0 + cb + i < NC; ++i)
                        out[i] = ubar[n0 + cb + i] + (double)v[i];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN)
                     : "memory");
}

// out[c][j] = in[j][c] for j < P, 0 for P <= j < Kp (W^T, K-major for the MMA).
__global__ void k_pad_transpose(const float* __restrict__ in, int P, int64_t NC, int Kp,
                                float* __restrict__ out) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = j0 + y;
        const int64_t c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (j < P && c < NC) ? in[(int64_t)j * NC + c] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t c = c0 + y;
        const int j = j0 + threadIdx.x;
        if (c < NC && j < Kp) out[c * Kp + j] = tile[threadIdx.x][y];
    }
}

}  // namespace

int guess_tc_k_padded(int P) { return (P + TK - 1) / TK * TK; }

void launch_pad_transpose(const float* W, int P, int64_t NC, int Kp, float* Wt, cudaStream_t st) {
    if (NC == 0) return;
    dim3 grid((unsigned)((NC + 31) / 32), (unsigned)((Kp + 31) / 32));
    k_pad_transpose<<<grid, dim3(32, 8), 0, st>>>(W, P, NC, Kp, Wt);
}

void launch_guess_tc(int64_t S, int64_t NC, int Kp, const float* psi, const float* Wt,
                     const double* ubar, double* U, int* err, cudaStream_t st) {
    if (S == 0 || NC == 0) return;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_guess_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        attr = true;
    }
    dim3 grid((unsigned)((NC + TN - 1) / TN), (unsigned)((S + TM - 1) / TM));
    k_guess_tc<<<grid, 128, SMEM_BYTES, st>>>(S, NC, Kp, psi, Wt, ubar, U, err);
}

}  // namespace klecgc
