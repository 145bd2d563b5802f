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

#include <float.h>

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

}  // namespace

qw_status launch_hash(const float *V, int64_t nv, int d, const float *A, const float *b, int m,
                      float w, int32_t *H, int64_t ld_row, int64_t ld_col, int *err,
                      unsigned long long *fixups, cudaStream_t s)
{
    if (nv == 0) return QW_OK;
    if (!((ld_row == m && ld_col == 1) || (ld_row == 1 && ld_col == nv))) return QW_ERR_ARG;
    dim3 grid((unsigned)((nv + BM - 1) / BM), (unsigned)((m + BN - 1) / BN));
    if (grid.x > 2147483647u) return QW_ERR_ARG;
    project_fp32_kernel<<<grid, NT, 0, s>>>(V, nv, d, A, b, m, w, H, ld_row, ld_col, err);
    QW_CUDA_TRY(cudaGetLastError());
    int64_t total = nv * (int64_t)m;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fixup_fp64_kernel<<<(unsigned)blocks, 256, 0, s>>>(V, nv, d, A, b, m, w, H, ld_row, ld_col,
                                                      err, fixups);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
