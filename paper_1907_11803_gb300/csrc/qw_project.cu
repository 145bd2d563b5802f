// qw_project.cu -- the projection step of the hash family (Section 3):
//   h_i(v) = floor((a_i . v + b_i) / w),   a_i ~ N(0, I), b_i ~ U[0, w).
//
// Pass 1 (FP32, tiled over rows x projections) computes t = a_i . v with FP32
// fused multiply-adds summed over j = 0..d-1 in order, then u = (t + b_i) / w
// with explicitly rounded FP32 operations.  Each fused multiply-add rounds
// once, and in a recursive sum the rounding errors add up without being
// amplified, so the error of t is at most u / (1 - u) * sum_j |s_j|, s_j the
// computed partial sums (u = 2^-24); that sum is accumulated in FP32 beside
// t and enlarged by (1 + 2 d u) * 1.01 for its own rounding.  (The a-priori
// bound gamma_d ||a_i|| ||v|| is typically ten times larger.)  Adding b and
// dividing by w add at most 2u |u| + u.  Whenever the distance of u to the
// nearest integer is not larger than that bound (or than 1e-5, i.e. 1e-5 w
// in projection units, whichever is larger), floor(u) is not trusted and the
// entry is marked.
//
// Pass 2 (FP64) recomputes every marked entry with the dot product summed in
// index order, each product and sum correctly rounded (no fused multiply-add),
// then (t + b) / w in double and floor: the same sequence of IEEE operations
// as the FP64 definition, so the bucket id equals it exactly.
#include "qw_internal.cuh"
#include "qw_tc.cuh"

#include <cuda_bf16.h>
#include <float.h>

#include <algorithm>

namespace qw {
namespace {

constexpr int BM = 64;   // rows per CTA
constexpr int BN = 64;   // projections per CTA
constexpr int BK = 32;   // dimension chunk
constexpr int NT = 256;  // threads

__global__ void __launch_bounds__(NT) project_fp32_kernel(
    const float *__restrict__ V, int64_t nv, int d, const float *__restrict__ A,
    const float *__restrict__ b, int m, float w, int32_t *__restrict__ H, int64_t ld_row,
    int64_t ld_col, int *__restrict__ err)
{
    __shared__ float Vs[BK][BM + 1];
    __shared__ float As[BK][BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid & 15;   // projection lane
    const int ty = tid >> 4;   // row lane
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int col0 = blockIdx.y * BN;

    float acc[4][4], run[4][4];  // partial sums and the sum of their magnitudes
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            acc[ii][jj] = 0.0f;
            run[ii][jj] = 0.0f;
        }

    for (int k0 = 0; k0 < d; k0 += BK) {
        // Stage a BM x BK block of V and a BN x BK block of A, transposed.
#pragma unroll
        for (int e = 0; e < (BM * BK) / NT; ++e) {
            int idx = tid + e * NT;
            int r = idx / BK, kk = idx % BK;
            int64_t gr = row0 + r;
            int gk = k0 + kk;
            Vs[kk][r] = (gr < nv && gk < d) ? V[gr * d + gk] : 0.0f;
            int gc = col0 + r;
            As[kk][r] = (gc < m && gk < d) ? A[(int64_t)gc * d + gk] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            float vr[4], ac[4];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) vr[ii] = Vs[kk][ty + 16 * ii];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) ac[jj] = As[kk][tx + 16 * jj];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    acc[ii][jj] = fmaf(vr[ii], ac[jj], acc[ii][jj]);
                    run[ii][jj] += fabsf(acc[ii][jj]);
                }
        }
        __syncthreads();
    }

    const float unit = 5.9604645e-08f;  // 2^-24
    // error of t per unit of the running magnitude sum, over w
    const float run_bound = unit * (1.0f + 2.0f * (float)d * unit) * 1.01f / w;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
        int64_t r = row0 + ty + 16 * ii;
        if (r >= nv) continue;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            int i = col0 + tx + 16 * jj;
            if (i >= m) continue;
            float u = __fdiv_rn(__fadd_rn(acc[ii][jj], b[i]), w);
            float f = floorf(u);
            int32_t h;
            if (!(f >= -2147483520.0f && f <= 2147483520.0f)) {
                // out of int32 (or NaN): let the FP64 pass decide and report
                h = kNeedsFp64;
            } else {
                float frac = u - f;                       // exact
                float near = fminf(frac, 1.0f - frac);
                float eps = fmaxf(run_bound * run[ii][jj] + 4.0f * unit * (fabsf(u) + 1.0f), 1e-5f);
                h = (near <= eps) ? kNeedsFp64 : (int32_t)f;
            }
            H[r * ld_row + (int64_t)i * ld_col] = h;
        }
    }
    (void)err;
}

// One thread per entry of the contiguous nv x m (row-major) or m x nv
// (projection-major) array; only marked entries do work.
__global__ void fixup_fp64_kernel(const float *__restrict__ V, int64_t nv, int d,
                                  const float *__restrict__ A, const float *__restrict__ b,
                                  int m, float w, int32_t *__restrict__ H, int64_t ld_row,
                                  int64_t ld_col, int *__restrict__ err,
                                  unsigned long long *__restrict__ fixups)
{
    const int64_t total = nv * (int64_t)m;
    unsigned long long mine = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t *hp = H + e;
        if (*hp != kNeedsFp64) continue;
        int64_t r, i;
        if (ld_col == 1) { r = e / m; i = e % m; }
        else { i = e / nv; r = e % nv; }
        const float *vr = V + r * (int64_t)d;
        const float *ar = A + i * (int64_t)d;
        double t = 0.0;
        for (int j = 0; j < d; ++j) t = __dadd_rn(t, __dmul_rn((double)ar[j], (double)vr[j]));
        double u = __ddiv_rn(__dadd_rn(t, (double)b[i]), (double)w);
        double f = floor(u);
        if (!(f >= -2147483647.0 && f <= 2147483646.0)) {
            atomicOr(err, 2);
            *hp = 0;
        } else {
            *hp = (int32_t)f;
        }
        ++mine;
    }
    if (fixups && mine) atomicAdd(fixups, mine);
}

// ---- the same projection on the tensor cores (tcgen05, BF16 in, FP32 out)
//
// Every FP32 input is split into two BF16 numbers, v = v_hi + v_lo + e with
// v_hi = bf16(v), v_lo = bf16(v - v_hi) (v - v_hi is exact in FP32) and
// |e| <= 2^-16 |v|; likewise a = a_hi + a_lo + e_a.  A CTA of 128 threads
// takes 128 rows and every projection; the three products that matter,
//   D_hh = X_hi A_hi^T,  D_hl = X_lo A_hi^T,  D_lh = X_hi A_lo^T,
// go to three FP32 accumulators in tensor memory (M = 128, N = m rounded up to
// 16, K = 16 per instruction, one issuing thread), and t = D_hh + (D_hl + D_lh)
// is formed in FP32 in the epilogue.  Error of t, for any order of the
// tensor cores' internal additions:
//   - dropped terms a_lo v_lo and those with e, e_a: <= 3.01 * 2^-16 S;
//   - accumulation, taking every addition inside the tensor core to lose at
//     most two units in the last place (2^-22 relative; rounding or
//     truncation): <= (d - 1) * 2^-22 * S for D_hh, and 2^-8 of that for the
//     two small accumulators;
//   - the two FP32 additions of the epilogue: <= 2^-23 S,
// with S = sum_j |a_j v_j| <= ||a|| ||v|| (Cauchy-Schwarz; norms formed in
// FP32 and enlarged by 1 %).  As in the CUDA-core pass, every entry whose
// value lies within that bound (and at least 1e-5 w) of a bucket edge is
// marked and recomputed in FP64 by fixup_fp64_kernel, so the bucket ids are
// those of the FP64 definition whatever the tensor cores' rounding.
constexpr int PT_ROWS = 128;  // rows per CTA (the MMA's M)
constexpr int PT_KC = 64;     // input coordinates per staged chunk

__global__ void __launch_bounds__(PT_ROWS, 1) project_tc_kernel(
    const float *__restrict__ V, int64_t nv, int d, const float *__restrict__ A,
    const float *__restrict__ b, int m, float w, int32_t *__restrict__ H, int64_t ld_row,
    int64_t ld_col, int *__restrict__ err, uint32_t ncols)
{
    extern __shared__ __align__(1024) unsigned char ptsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase_s;
    __shared__ int s_stuck;
    __shared__ float vnorm2[PT_ROWS], anorm2[128];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int N = (m + 15) & ~15;                      // projections, padded
    unsigned char *xhi = ptsm;                         // 128 x PT_KC BF16
    unsigned char *xlo = xhi + PT_ROWS * PT_KC * 2;
    unsigned char *ahi = xlo + PT_ROWS * PT_KC * 2;    // N x PT_KC BF16
    unsigned char *alo = ahi + 128 * PT_KC * 2;
    const int64_t r0 = (int64_t)blockIdx.x * PT_ROWS;
    if (tid == 0) {
        s_stuck = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    vnorm2[tid] = 0.0f;
    anorm2[tid] = 0.0f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem(&tbase_s)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tbase_s;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t idesc = tc_idesc_bf16(PT_ROWS, N);
    uint32_t phase = 0;
    // split a float into BF16 hi + lo
    auto split = [](float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
        hi = __float2bfloat16_rn(v);
        lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    };
    for (int k0 = 0; k0 < d; k0 += PT_KC) {
        // stage the chunk: rows of V (4 consecutive coordinates per piece)
        for (int p = tid; p < PT_ROWS * (PT_KC / 4); p += PT_ROWS) {
            const int r = p / (PT_KC / 4), c = (p % (PT_KC / 4)) * 4;
            const int64_t gr = r0 + r;
            __align__(8) __nv_bfloat16 h4[4], l4[4];
            float sq = 0.0f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int gc = k0 + c + u;
                const float v = (gr < nv && gc < d) ? V[gr * d + gc] : 0.0f;
                sq = fmaf(v, v, sq);
                split(v, h4[u], l4[u]);
            }
            if (sq != 0.0f) atomicAdd(&vnorm2[r], sq);
            *reinterpret_cast<uint2 *>(xhi + tc_off(r, c, PT_KC)) = *reinterpret_cast<const uint2 *>(h4);
            *reinterpret_cast<uint2 *>(xlo + tc_off(r, c, PT_KC)) = *reinterpret_cast<const uint2 *>(l4);
        }
        // and rows of A (projections past m are zero)
        for (int p = tid; p < N * (PT_KC / 4); p += PT_ROWS) {
            const int r = p / (PT_KC / 4), c = (p % (PT_KC / 4)) * 4;
            __align__(8) __nv_bfloat16 h4[4], l4[4];
            float sq = 0.0f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int gc = k0 + c + u;
                const float v = (r < m && gc < d) ? A[(int64_t)r * d + gc] : 0.0f;
                sq = fmaf(v, v, sq);
                split(v, h4[u], l4[u]);
            }
            if (sq != 0.0f) atomicAdd(&anorm2[r], sq);
            *reinterpret_cast<uint2 *>(ahi + tc_off(r, c, PT_KC)) = *reinterpret_cast<const uint2 *>(h4);
            *reinterpret_cast<uint2 *>(alo + tc_off(r, c, PT_KC)) = *reinterpret_cast<const uint2 *>(l4);
        }
        tc_fence_async_smem();
        tc_fence_before();
        __syncthreads();
        const bool go = s_stuck == 0;
        if (tid == 0 && go) {
            tc_fence_after();
#pragma unroll
            for (int s2 = 0; s2 < PT_KC / 16; ++s2) {
                const uint32_t acc = (k0 | s2) != 0 ? 1u : 0u;
                const uint32_t kb = (uint32_t)(2 * s2) * 128;  // 16 k = two core matrices
                const uint64_t dxh = tc_desc(xhi + kb, 128, PT_KC * 16);
                const uint64_t dxl = tc_desc(xlo + kb, 128, PT_KC * 16);
                const uint64_t dah = tc_desc(ahi + kb, 128, PT_KC * 16);
                const uint64_t dal = tc_desc(alo + kb, 128, PT_KC * 16);
                tc_mma(tbase, dxh, dah, idesc, acc);                    // X_hi A_hi^T
                tc_mma(tbase + (uint32_t)N, dxl, dah, idesc, acc);      // X_lo A_hi^T
                tc_mma(tbase + 2u * (uint32_t)N, dxh, dal, idesc, acc); // X_hi A_lo^T
            }
            tc_commit(&bar);
        }
        if (go) {
            if (!tc_wait(&bar, phase)) s_stuck = 1;
            phase ^= 1;
        }
        tc_fence_after();
        __syncthreads();  // the chunk buffers are rewritten next
    }
    // epilogue: row = thread
    const int64_t r = r0 + tid;
    const bool stuck = s_stuck != 0;
    const float unit = 5.9604645e-08f;  // 2^-24
    const float vn = sqrtf(vnorm2[tid]) * 1.01f;
    const float cacc = (3.01f * 1.52587890625e-05f                 // 3.01 * 2^-16
                        + (float)(d > 1 ? d - 1 : 0) * 2.384185791e-07f * 1.01f  // (d-1) 2^-22
                        + 2.0f * unit) * 1.01f;
    for (int n0 = 0; n0 < N; n0 += 16) {
        float hh[16], hl[16], lh[16];
        tc_ld16(tbase + lane_base + (uint32_t)n0, hh);
        tc_ld16(tbase + lane_base + (uint32_t)(N + n0), hl);
        tc_ld16(tbase + lane_base + (uint32_t)(2 * N + n0), lh);
        if (r >= nv) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int i = n0 + j;
            if (i >= m) continue;
            const float t = __fadd_rn(hh[j], __fadd_rn(hl[j], lh[j]));
            const float u = __fdiv_rn(__fadd_rn(t, b[i]), w);
            const float f = floorf(u);
            int32_t h;
            if (stuck || !(f >= -2147483520.0f && f <= 2147483520.0f)) {
                h = kNeedsFp64;  // out of int32, NaN, or a wait that gave up: FP64 decides
            } else {
                const float frac = u - f;
                const float near = fminf(frac, 1.0f - frac);
                const float an = sqrtf(anorm2[i]) * 1.01f;
                const float eps = fmaxf(cacc * an * vn / w + 4.0f * unit * (fabsf(u) + 1.0f), 1e-5f);
                h = (near <= eps) ? kNeedsFp64 : (int32_t)f;
            }
            H[r * ld_row + (int64_t)i * ld_col] = h;
        }
    }
    if (tid == 0 && stuck) atomicOr(err, 16);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(ncols)
                     : "memory");
    }
}

}  // namespace

qw_status launch_hash(const float *V, int64_t nv, int d, const float *A, const float *b, int m,
                      float w, int32_t *H, int64_t ld_row, int64_t ld_col, int *err,
                      unsigned long long *fixups, cudaStream_t s, bool tensor_cores)
{
    if (nv == 0) return QW_OK;
    if (!((ld_row == m && ld_col == 1) || (ld_row == 1 && ld_col == nv))) return QW_ERR_ARG;
    if (tensor_cores && m <= 128) {
        const int N = (m + 15) & ~15;
        uint32_t ncols = 32;
        while (ncols < (uint32_t)(3 * N)) ncols <<= 1;
        // shared memory sized so that the CTAs resident on an SM never ask
        // for more than its 512 TMEM columns (no allocation waits)
        const size_t per = (size_t)(2 * PT_ROWS + 2 * 128) * PT_KC * 2;
        const size_t smem = std::max<size_t>(per, ncols > 256 ? (size_t)120 << 10 : (size_t)80 << 10);
        QW_CUDA_TRY(cudaFuncSetAttribute(project_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int64_t blocks = (nv + PT_ROWS - 1) / PT_ROWS;
        if (blocks > 2147483647LL) return QW_ERR_ARG;
        project_tc_kernel<<<(unsigned)blocks, PT_ROWS, smem, s>>>(V, nv, d, A, b, m, w, H, ld_row,
                                                                  ld_col, err, ncols);
        QW_CUDA_TRY(cudaGetLastError());
    } else {
        dim3 grid((unsigned)((nv + BM - 1) / BM), (unsigned)((m + BN - 1) / BN));
        if (grid.x > 2147483647u) return QW_ERR_ARG;
        project_fp32_kernel<<<grid, NT, 0, s>>>(V, nv, d, A, b, m, w, H, ld_row, ld_col, err);
        QW_CUDA_TRY(cudaGetLastError());
    }
    int64_t total = nv * (int64_t)m;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fixup_fp64_kernel<<<(unsigned)blocks, 256, 0, s>>>(V, nv, d, A, b, m, w, H, ld_row, ld_col,
                                                      err, fixups);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
