// qw_mlp.cu -- the learned part: a small multilayer perceptron that predicts,
// from a query's features, the level at which the collision-counting loop
// stops, so the level path can begin at a later level (a query that then
// stops at its first level is recomputed from level 0: the prediction changes
// only the speed, never the result).
//
// The paper trains an offline model to pick its cache split (Section 5.2); it
// gives no network.  This one is x (n_in) -> ReLU(W1 x + b1) -> ReLU(W2 . + b2)
// -> W3 . + b3 (C logits), trained with mean softmax cross-entropy and Adam.
// Weights are used as FP16 copies of FP32 master weights; every product is
// accumulated in FP32.  Training (forward, backward, the optimizer step) runs
// on tiled CUDA-core GEMMs, once and outside the query path.  The forward
// pass of the query path (the first levels of a workload's queries) runs on
// the tensor cores (mlp_forward_tc_kernel: tcgen05.mma, accumulators in tensor
// memory) when the network has its shape, else on the fused CUDA-core kernel
// start_model_kernel.
#include "qw_internal.cuh"
#include "qw_tc.cuh"

#include <cuda_fp16.h>

#include <algorithm>
#include <string>
#include <vector>

namespace qw {
namespace {

constexpr int GM = 64, GN = 64, GK = 16, GT = 256;

template <typename TB>
__device__ __forceinline__ float to_f(TB v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) with arbitrary strides.
// EPI 0: store; 1: add bias; 2: add bias, store pre-activation to C and
// ReLU(.) to Aout.
template <typename TB, int EPI>
__global__ void __launch_bounds__(GT) mlp_gemm_kernel(int M, int N, int K,
                                                      const float *__restrict__ A, int64_t sam,
                                                      int64_t sak, const TB *__restrict__ B,
                                                      int64_t sbk, int64_t sbn,
                                                      float *__restrict__ C, int64_t ldc,
                                                      const float *__restrict__ bias,
                                                      float *__restrict__ Aout)
{
    __shared__ float As[GK][GM + 1];
    __shared__ float Bs[GK][GN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GM * GK; e += GT) {
            const int mm = e / GK, kk = e % GK;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.0f;
        }
        for (int e = threadIdx.x; e < GN * GK; e += GT) {
            const int nn = e / GK, kk = e % GK;
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < K) ? to_f<TB>(B[gk * sbk + gn * sbn]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            float v = acc[i][j];
            if (EPI >= 1) v += bias[gn];
            C[gm * ldc + gn] = v;
            if (EPI == 2) Aout[gm * ldc + gn] = v > 0.0f ? v : 0.0f;
        }
    }
}

// Softmax cross-entropy of one row per warp: adds -log p[y] to *loss_sum and
// writes d logits = (p - onehot(y)) * inv_n; or, without labels, p.
__global__ void softmax_rows_kernel(const float *__restrict__ Z, int n, int C,
                                    const int32_t *__restrict__ y, float inv_n,
                                    float *__restrict__ dZ, float *__restrict__ loss_sum,
                                    float *__restrict__ prob)
{
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *z = Z + (int64_t)r * C;
    float mx = -INFINITY;
    for (int c = lane; c < C; c += 32) mx = fmaxf(mx, z[c]);
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    float s = 0.0f;
    for (int c = lane; c < C; c += 32) s += __expf(z[c] - mx);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const float inv_s = 1.0f / s;
    for (int c = lane; c < C; c += 32) {
        const float p = __expf(z[c] - mx) * inv_s;
        if (prob) prob[(int64_t)r * C + c] = p;
        if (dZ) dZ[(int64_t)r * C + c] = (p - ((y && c == y[r]) ? 1.0f : 0.0f)) * inv_n;
    }
    if (lane == 0 && y && loss_sum) {
        const float logp = (z[y[r]] - mx) - __logf(s);
        atomicAdd(loss_sum, -logp);
    }
}

// out[c] = sum_r D[r][c]
__global__ void colsum_kernel(const float *__restrict__ D, int n, int C, float *__restrict__ out)
{
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s += D[(int64_t)r * C + c];
    __shared__ float red[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (int)(blockDim.x / 32) ? red[threadIdx.x] : 0.0f;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) out[c] = s;
    }
}

__global__ void relu_back_kernel(float *__restrict__ dA, const float *__restrict__ Z, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!(Z[i] > 0.0f)) dA[i] = 0.0f;
}

__global__ void to_half_kernel(const float *__restrict__ p, __half *__restrict__ h, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        h[i] = __float2half_rn(p[i]);
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m1, float *__restrict__ m2,
                            __half *__restrict__ h, int64_t count, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gi;
        const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        const float v = p[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        p[i] = v;
        h[i] = __float2half_rn(v);
    }
}

// Start level of every query: the largest s whose predicted probability of
// stopping at a level <= s is at most eps (0 when none is).
__global__ void start_level_kernel(const float *__restrict__ prob, int n, int C, float eps,
                                   int32_t *__restrict__ start)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float cdf = 0.0f;
    int s = 0;
    for (int c = 0; c < C - 1; ++c) {
        cdf += prob[(int64_t)q * C + c];
        if (cdf <= eps) s = c + 1; else break;
    }
    // s - 1 is the last level with cdf <= eps; a start beyond it risks a
    // stop at the start level
    start[q] = s > 0 ? s - 1 : 0;
}

// Features of a query: its coordinates scaled by 1 / (data RMS), then for
// every projection its position in the data's bucket-id range.
__global__ void features_kernel(const float *__restrict__ Q, const int32_t *__restrict__ HQ,
                                int64_t nq, int d, int m, const int32_t *__restrict__ o,
                                const int32_t *__restrict__ span, float xs,
                                float *__restrict__ F)
{
    const int64_t q = blockIdx.x;
    if (q >= nq) return;
    const int nin = d + m;
    for (int j = threadIdx.x; j < d; j += blockDim.x) F[q * nin + j] = Q[q * d + j] * xs;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double g = (double)HQ[q * m + i] - (double)o[i];
        double pos = (g + 0.5) / ((double)span[i] + 1.0);
        pos = pos < -1.0 ? -1.0 : (pos > 2.0 ? 2.0 : pos);
        F[q * nin + d + i] = (float)(pos - 0.5);
    }
}

__global__ void sumsq_kernel(const float *__restrict__ X, int64_t count, double *__restrict__ out)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (double)X[i] * (double)X[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

template <typename TB, int EPI>
qw_status gemm(int M, int N, int K, const float *A, int64_t sam, int64_t sak, const TB *B,
               int64_t sbk, int64_t sbn, float *C, int64_t ldc, const float *bias, float *Aout,
               cudaStream_t s)
{
    if (M <= 0 || N <= 0) return QW_OK;
    dim3 grid((unsigned)((N + GN - 1) / GN), (unsigned)((M + GM - 1) / GM));
    mlp_gemm_kernel<TB, EPI><<<grid, GT, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias,
                                                 Aout);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace
}  // namespace qw

using namespace qw;

struct qw_mlp {
    int n_in = 0, H = 0, C = 0;
    int64_t np = 0;
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    DevBuf p32, p16, grad, m1, m2, work, scalar;
    DevBuf p16t;  // k-major FP16 copies of W1, W2, W3 for the fused inference kernel
    DevBuf tc_err;  // error word of the tensor-core forward pass
    int cap = 0;  // rows the work buffers hold
    int64_t step = 0;
    int64_t version = 0, t_version = -1;  // weights changed / k-major copies made at

    float *Z1, *A1, *Z2, *A2, *Z3, *D3, *DA, *DZ;

    qw_status ensure_work(int rows)
    {
        if (rows <= cap) return QW_OK;
        const size_t per = (size_t)rows;
        const size_t bytes = per * (6 * (size_t)H + 2 * (size_t)C) * sizeof(float);
        QW_TRY(work.ensure(bytes));
        float *p = work.as<float>();
        Z1 = p; p += per * H;
        A1 = p; p += per * H;
        Z2 = p; p += per * H;
        A2 = p; p += per * H;
        DA = p; p += per * H;
        DZ = p; p += per * H;
        Z3 = p; p += per * C;
        D3 = p;
        cap = rows;
        return QW_OK;
    }

    // forward of rows [0, n) of X (n <= cap): logits in Z3
    qw_status forward(const float *X, int n, cudaStream_t s)
    {
        const __half *h = p16.as<__half>();
        const float *p = p32.as<float>();
        QW_TRY((gemm<__half, 2>(n, H, n_in, X, n_in, 1, h + oW1, 1, n_in, Z1, H, p + ob1, A1, s)));
        QW_TRY((gemm<__half, 2>(n, H, H, A1, H, 1, h + oW2, 1, H, Z2, H, p + ob2, A2, s)));
        QW_TRY((gemm<__half, 1>(n, C, H, A2, H, 1, h + oW3, 1, H, Z3, C, p + ob3, nullptr, s)));
        return QW_OK;
    }

    // loss sum into scalar[0] and gradient (mean over n rows) into grad
    qw_status backward(const float *X, const int32_t *y, int n, cudaStream_t s)
    {
        const __half *h = p16.as<__half>();
        float *g = grad.as<float>();
        float *loss = scalar.as<float>();
        softmax_rows_kernel<<<(n + 7) / 8, 256, 0, s>>>(Z3, n, C, y, 1.0f / (float)n, D3, loss,
                                                        nullptr);
        QW_CUDA_TRY(cudaGetLastError());
        // layer 3
        QW_TRY((gemm<float, 0>(C, H, n, D3, 1, C, A2, H, 1, g + oW3, H, nullptr, nullptr, s)));
        colsum_kernel<<<C, 256, 0, s>>>(D3, n, C, g + ob3);
        QW_CUDA_TRY(cudaGetLastError());
        QW_TRY((gemm<__half, 0>(n, H, C, D3, C, 1, h + oW3, H, 1, DA, H, nullptr, nullptr, s)));
        relu_back_kernel<<<152 * 4, 256, 0, s>>>(DA, Z2, (int64_t)n * H);
        QW_CUDA_TRY(cudaGetLastError());
        // layer 2 (DA now holds d Z2)
        QW_TRY((gemm<float, 0>(H, H, n, DA, 1, H, A1, H, 1, g + oW2, H, nullptr, nullptr, s)));
        colsum_kernel<<<H, 256, 0, s>>>(DA, n, H, g + ob2);
        QW_CUDA_TRY(cudaGetLastError());
        QW_TRY((gemm<__half, 0>(n, H, H, DA, H, 1, h + oW2, H, 1, DZ, H, nullptr, nullptr, s)));
        relu_back_kernel<<<152 * 4, 256, 0, s>>>(DZ, Z1, (int64_t)n * H);
        QW_CUDA_TRY(cudaGetLastError());
        // layer 1 (DZ holds d Z1)
        QW_TRY((gemm<float, 0>(H, n_in, n, DZ, 1, H, X, n_in, 1, g + oW1, n_in, nullptr, nullptr,
                               s)));
        colsum_kernel<<<H, 256, 0, s>>>(DZ, n, H, g + ob1);
        QW_CUDA_TRY(cudaGetLastError());
        return QW_OK;
    }
};

static qw_status mlp_error(const char *msg)
{
    set_error(std::string("qw_mlp: ") + msg);
    return QW_ERR_ARG;
}

extern "C" {

qw_status qw_mlp_create(int32_t n_in, int32_t hidden, int32_t classes, qw_mlp **out)
{
    clear_error();
    if (!out) return mlp_error("out is null");
    *out = nullptr;
    if (n_in < 1 || hidden < 1 || classes < 2 || n_in > 65536 || hidden > 65536 || classes > 1024)
        return mlp_error("bad layer sizes");
    qw_mlp *mp = new (std::nothrow) qw_mlp();
    if (!mp) return QW_ERR_OOM;
    mp->n_in = n_in;
    mp->H = hidden;
    mp->C = classes;
    int64_t o = 0;
    mp->oW1 = o; o += (int64_t)hidden * n_in;
    mp->ob1 = o; o += hidden;
    mp->oW2 = o; o += (int64_t)hidden * hidden;
    mp->ob2 = o; o += hidden;
    mp->oW3 = o; o += (int64_t)classes * hidden;
    mp->ob3 = o; o += classes;
    mp->np = o;
    qw_status st = QW_OK;
    if ((st = mp->p32.ensure(o * 4)) != QW_OK || (st = mp->p16.ensure(o * 2)) != QW_OK ||
        (st = mp->grad.ensure(o * 4)) != QW_OK || (st = mp->m1.ensure(o * 4)) != QW_OK ||
        (st = mp->m2.ensure(o * 4)) != QW_OK || (st = mp->scalar.ensure(64)) != QW_OK) {
        delete mp;
        return st;
    }
    cudaMemset(mp->p32.p, 0, o * 4);
    cudaMemset(mp->p16.p, 0, o * 2);
    cudaMemset(mp->m1.p, 0, o * 4);
    cudaMemset(mp->m2.p, 0, o * 4);
    *out = mp;
    return QW_OK;
}

int64_t qw_mlp_param_count(const qw_mlp *mp) { return mp ? mp->np : -1; }

qw_status qw_mlp_set_params(qw_mlp *mp, const float *params, int64_t count)
{
    clear_error();
    if (!mp || !params) return mlp_error("null pointer");
    if (count != mp->np) return mlp_error("parameter count mismatch");
    QW_CUDA_TRY(cudaMemcpy(mp->p32.p, params, count * 4, cudaMemcpyHostToDevice));
    to_half_kernel<<<152 * 4, 256>>>(mp->p32.as<float>(), mp->p16.as<__half>(), count);
    mp->version += 1;
    QW_CUDA_TRY(cudaGetLastError());
    QW_CUDA_TRY(cudaMemset(mp->m1.p, 0, count * 4));
    QW_CUDA_TRY(cudaMemset(mp->m2.p, 0, count * 4));
    mp->step = 0;
    QW_CUDA_TRY(cudaDeviceSynchronize());
    return QW_OK;
}

qw_status qw_mlp_get_params(const qw_mlp *mp, float *params, int64_t count)
{
    clear_error();
    if (!mp || !params) return mlp_error("null pointer");
    if (count != mp->np) return mlp_error("parameter count mismatch");
    QW_CUDA_TRY(cudaDeviceSynchronize());
    QW_CUDA_TRY(cudaMemcpy(params, mp->p32.p, count * 4, cudaMemcpyDeviceToHost));
    return QW_OK;
}

qw_status qw_mlp_loss_grad(qw_mlp *mp, const float *X, const int32_t *y, int64_t n, float *loss,
                           float *grad, void *stream)
{
    clear_error();
    if (!mp || !X || !y) return mlp_error("null pointer");
    if (n < 1 || n > (1 << 20)) return mlp_error("n out of range");
    cudaStream_t s = (cudaStream_t)stream;
    QW_TRY(mp->ensure_work((int)n));
    QW_CUDA_TRY(cudaMemsetAsync(mp->scalar.p, 0, 64, s));
    QW_TRY(mp->forward(X, (int)n, s));
    QW_TRY(mp->backward(X, y, (int)n, s));
    float ls = 0.0f;
    QW_CUDA_TRY(cudaMemcpyAsync(&ls, mp->scalar.p, 4, cudaMemcpyDeviceToHost, s));
    if (grad)
        QW_CUDA_TRY(cudaMemcpyAsync(grad, mp->grad.p, mp->np * 4, cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    if (loss) *loss = ls / (float)n;
    return QW_OK;
}

qw_status qw_mlp_train(qw_mlp *mp, const float *X, const int32_t *y, int64_t n, int32_t epochs,
                       int32_t batch, float lr, float *final_loss, void *stream)
{
    clear_error();
    if (!mp || !X || !y) return mlp_error("null pointer");
    if (n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f)) return mlp_error("bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int B = (int)std::min<int64_t>(batch, n);
    QW_TRY(mp->ensure_work(B));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float last = 0.0f;
    for (int ep = 0; ep < epochs; ++ep) {
        QW_CUDA_TRY(cudaMemsetAsync(mp->scalar.p, 0, 64, s));
        for (int64_t r0 = 0; r0 < n; r0 += B) {
            const int nb = (int)std::min<int64_t>(B, n - r0);
            const float *Xb = X + r0 * mp->n_in;
            QW_TRY(mp->forward(Xb, nb, s));
            QW_TRY(mp->backward(Xb, y + r0, nb, s));
            mp->step += 1;
            mp->version += 1;
            const float c1 = 1.0f - powf(b1, (float)mp->step);
            const float c2 = 1.0f - powf(b2, (float)mp->step);
            adam_kernel<<<152 * 4, 256, 0, s>>>(mp->p32.as<float>(), mp->grad.as<float>(),
                                                mp->m1.as<float>(), mp->m2.as<float>(),
                                                mp->p16.as<__half>(), mp->np, lr, b1, b2, eps, c1,
                                                c2);
            QW_CUDA_TRY(cudaGetLastError());
        }
        float ls = 0.0f;
        QW_CUDA_TRY(cudaMemcpyAsync(&ls, mp->scalar.p, 4, cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        last = ls / (float)n;
    }
    if (final_loss) *final_loss = last;
    return QW_OK;
}

qw_status qw_mlp_predict(qw_mlp *mp, const float *X, int64_t n, float *prob, void *stream)
{
    clear_error();
    if (!mp || !X || !prob) return mlp_error("null pointer");
    if (n < 0) return mlp_error("n < 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int B = 1024;
    QW_TRY(mp->ensure_work(B));
    for (int64_t r0 = 0; r0 < n; r0 += B) {
        const int nb = (int)std::min<int64_t>(B, n - r0);
        QW_TRY(mp->forward(X + r0 * mp->n_in, nb, s));
        softmax_rows_kernel<<<(nb + 7) / 8, 256, 0, s>>>(mp->Z3, nb, mp->C, nullptr, 1.0f, nullptr,
                                                         nullptr, prob + r0 * mp->C);
        QW_CUDA_TRY(cudaGetLastError());
    }
    return QW_OK;
}

void qw_mlp_free(qw_mlp *mp)
{
    if (!mp) return;
    cudaDeviceSynchronize();
    delete mp;
}

}  // extern "C"

namespace qw {

int mlp_inputs(const qw_mlp *mp) { return mp ? mp->n_in : 0; }
int mlp_classes(const qw_mlp *mp) { return mp ? mp->C : 0; }

namespace {

// out[k * rows + j] = in[j * cols + k] (a rows x cols matrix made k-major).
__global__ void transpose_half_kernel(const __half *__restrict__ in, int rows, int cols,
                                      __half *__restrict__ out)
{
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / cols, k = e % cols;
        out[k * rows + j] = in[e];
    }
}

constexpr int SM_RB = 16;  // queries per block of the fused inference kernel
constexpr int SM_THREADS = 256;
static_assert(SM_RB % 8 == 0, "two halves of the rows, four per float4");

// Out[j][r] = ReLU(b[j] + sum_k In[k][r] Wt[k][j]) for the block's SM_RB rows
// (In, Out in shared memory, k-major; Wt: K x N FP16).  Thread t computes the
// neuron pair (2p, 2p + 1), p = t mod (SM_THREADS / 2), for half of the rows,
// reading both weights with one 4-byte load (N even; an odd last neuron takes
// the pair's first half) and keeping eight k steps of weights in flight.
__device__ __forceinline__ void dense_relu(const float *In, int K, const __half *__restrict__ Wt,
                                           const float *__restrict__ b, int N, float *Out)
{
    constexpr int PAIRS = SM_THREADS / 2;
    constexpr int RH = SM_RB / 2;  // rows per thread
    const int rh = threadIdx.x / PAIRS;
    // pairs load as one __half2 when every pair starts 4-byte aligned
    const bool even = (N & 1) == 0 && (reinterpret_cast<uintptr_t>(Wt) & 3u) == 0;
    for (int p = threadIdx.x % PAIRS; 2 * p < N; p += PAIRS) {
        const int j = 2 * p;
        const bool two = j + 1 < N;
        float acc0[RH], acc1[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            acc0[r] = b[j];
            acc1[r] = two ? b[j + 1] : 0.0f;
        }
        int k = 0;
        for (; k + 8 <= K; k += 8) {
            float2 w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const __half *wp = Wt + (int64_t)(k + u) * N + j;
                if (even) {
                    w[u] = __half22float2(*reinterpret_cast<const __half2 *>(wp));
                } else {
                    w[u].x = __half2float(wp[0]);
                    w[u].y = two ? __half2float(wp[1]) : 0.0f;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 *x4 = reinterpret_cast<const float4 *>(In + (k + u) * SM_RB + rh * RH);
#pragma unroll
                for (int r4 = 0; r4 < RH / 4; ++r4) {
                    const float4 x = x4[r4];
                    acc0[4 * r4 + 0] = fmaf(x.x, w[u].x, acc0[4 * r4 + 0]);
                    acc0[4 * r4 + 1] = fmaf(x.y, w[u].x, acc0[4 * r4 + 1]);
                    acc0[4 * r4 + 2] = fmaf(x.z, w[u].x, acc0[4 * r4 + 2]);
                    acc0[4 * r4 + 3] = fmaf(x.w, w[u].x, acc0[4 * r4 + 3]);
                    acc1[4 * r4 + 0] = fmaf(x.x, w[u].y, acc1[4 * r4 + 0]);
                    acc1[4 * r4 + 1] = fmaf(x.y, w[u].y, acc1[4 * r4 + 1]);
                    acc1[4 * r4 + 2] = fmaf(x.z, w[u].y, acc1[4 * r4 + 2]);
                    acc1[4 * r4 + 3] = fmaf(x.w, w[u].y, acc1[4 * r4 + 3]);
                }
            }
        }
        for (; k < K; ++k) {
            const float w0 = __half2float(Wt[(int64_t)k * N + j]);
            const float w1 = two ? __half2float(Wt[(int64_t)k * N + j + 1]) : 0.0f;
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const float x = In[k * SM_RB + rh * RH + r];
                acc0[r] = fmaf(x, w0, acc0[r]);
                acc1[r] = fmaf(x, w1, acc1[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            Out[j * SM_RB + rh * RH + r] = fmaxf(acc0[r], 0.0f);
            if (two) Out[(j + 1) * SM_RB + rh * RH + r] = fmaxf(acc1[r], 0.0f);
        }
    }
}

// The start model's inference for SM_RB queries per block, in one launch:
// the features (as features_kernel), the three layers with FP16 weights and
// FP32 accumulation, the softmax, and the first-level rule: with s the first
// level whose predicted probability of stopping at or before it exceeds eps,
// start at s - shift (shift 1: one level early, so the previous level is
// counted; shift 0: at s itself, where the previous level's candidates are
// recounted afterwards).  The prediction only chooses where a query starts,
// so its rounding cannot change any result.
__global__ void __launch_bounds__(SM_THREADS) start_model_kernel(
    const float *__restrict__ Q, const int32_t *__restrict__ HQ, int nq, int d, int m,
    const int32_t *__restrict__ o, const int32_t *__restrict__ span, float xs,
    const __half *__restrict__ W1t, const float *__restrict__ b1, const __half *__restrict__ W2t,
    const float *__restrict__ b2, const __half *__restrict__ W3t, const float *__restrict__ b3,
    int H, int C, float eps, int shift, int32_t *__restrict__ start)
{
    extern __shared__ __align__(16) float smf[];
    const int nin = d + m;
    float *X = smf;                   // nin x SM_RB (k-major)
    float *A1 = X + nin * SM_RB;      // H x SM_RB
    float *A2 = A1 + H * SM_RB;       // H x SM_RB
    float *Z = A2 + H * SM_RB;        // SM_RB x C
    const int r0 = blockIdx.x * SM_RB;
    const int rows = min(SM_RB, nq - r0);
    for (int e = threadIdx.x; e < SM_RB * nin; e += SM_THREADS) {
        const int r = e / nin, j = e % nin;
        float v = 0.0f;
        if (r < rows) {
            const int64_t q = r0 + r;
            if (j < d) {
                v = Q[q * d + j] * xs;
            } else {
                const int i = j - d;
                const double g = (double)HQ[q * m + i] - (double)o[i];
                double pos = (g + 0.5) / ((double)span[i] + 1.0);
                pos = pos < -1.0 ? -1.0 : (pos > 2.0 ? 2.0 : pos);
                v = (float)(pos - 0.5);
            }
        }
        X[j * SM_RB + r] = v;
    }
    __syncthreads();
    dense_relu(X, nin, W1t, b1, H, A1);
    __syncthreads();
    dense_relu(A1, H, W2t, b2, H, A2);
    __syncthreads();
    for (int e = threadIdx.x; e < SM_RB * C; e += SM_THREADS) {
        const int r = e / C, c = e % C;
        float z = b3[c];
        for (int k = 0; k < H; ++k) z = fmaf(A2[k * SM_RB + r], __half2float(W3t[(int64_t)k * C + c]), z);
        Z[r * C + c] = z;
    }
    __syncthreads();
    if ((int)threadIdx.x < rows) {
        const float *z = Z + threadIdx.x * C;
        float mx = -INFINITY;
        for (int c = 0; c < C; ++c) mx = fmaxf(mx, z[c]);
        float sum = 0.0f;
        for (int c = 0; c < C; ++c) sum += __expf(z[c] - mx);
        const float inv = 1.0f / sum;
        float cdf = 0.0f;
        int s = 0;
        for (int c = 0; c < C - 1; ++c) {
            cdf += __expf(z[c] - mx) * inv;
            if (cdf <= eps) s = c + 1; else break;
        }
        start[r0 + threadIdx.x] = s > shift ? s - shift : 0;
    }
}

// ---- the same forward pass on the fifth-generation tensor cores (tcgen05)
//
// One CTA of 128 threads answers 128 rows.  The layers are chained GEMMs
// [128 x K] x [K x N]: the activations (FP16) are the A operand in shared
// memory, the FP16 weight copies (row-major N x K, i.e. K-major) are the B
// operand, streamed through shared memory 64 k at a time, and the FP32
// accumulators live in tensor memory (TMEM): layer 1 in columns [0, 256),
// layer 2 in [256, 512), layer 3 again from column 0.  One thread issues the
// tcgen05.mma instructions (M = 128, N = the layer's width, K = 16 each) and
// commits them to an mbarrier; after the (bounded) wait, warp w reads TMEM
// lanes 32w .. 32w + 31, i.e. row = thread, adds the bias, applies ReLU and
// writes the next layer's A operand.  Operands use the no-swizzle K-major
// layout of 8-row x 16-byte core matrices: core matrix (i, j) (rows 8i..8i+7,
// k 8j..8j+7) at byte (i * K / 8 + j) * 128 of the tile, so core matrices
// adjacent in k are 128 bytes apart (the descriptor's leading-dimension
// offset) and adjacent in rows K * 16 bytes apart (its stride offset).
constexpr int TC_ROWS = 128;
constexpr int TC_KC = 64;          // k per weight chunk
constexpr int TC_MAXN = 256;       // widest layer
constexpr int TC_MAXK = 576;       // widest input (d + m)
constexpr int TC_MAXC = 32;        // classes

// Rows' inputs: X (n x K0 FP32, the features) when X is given, else the
// features of queries Q / HQ as start_model_kernel forms them.  Output: the
// class probabilities (prob, n x C) when prob is given, else each row's first
// level (start_model_kernel's rule).  W1, W2, W3: FP16, row-major (N x K).
// err (optional): bit 16 set when a wait gave up (rows then get level 0 or NaN).
// A CTA answers `rows` <= 128 rows (the MMA tiles stay 128 high, the rest
// zero), so that small workloads still spread over every SM.
__global__ void __launch_bounds__(TC_ROWS, 1) mlp_forward_tc_kernel(
    const float *__restrict__ X, const float *__restrict__ Q, const int32_t *__restrict__ HQ,
    int n, int rows, int d, int m, const int32_t *__restrict__ o, const int32_t *__restrict__ span, float xs,
    int K0, const __half *__restrict__ W1, const float *__restrict__ b1,
    const __half *__restrict__ W2, const float *__restrict__ b2, const __half *__restrict__ W3,
    const float *__restrict__ b3, int H, int C, float *__restrict__ prob, float eps, int shift,
    int32_t *__restrict__ start, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase_s;
    __shared__ int s_stuck;
    const int Ka = K0 > H ? K0 : H;
    unsigned char *act = tsm;                                  // 128 x Ka FP16
    unsigned char *wb = tsm + (size_t)TC_ROWS * Ka * 2;       // 256 x 64 FP16
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    if (tid == 0) {
        s_stuck = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         tc_smem(&tbase_s))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the first layer's input in FP16
    for (int e = tid; e < TC_ROWS * K0; e += TC_ROWS) {
        const int r = e / K0, j = e - r * K0;
        const int64_t q = r0 + r;
        float v = 0.0f;
        if (r < rows && q < n) {
            if (X) {
                v = X[q * K0 + j];
            } else if (j < d) {
                v = Q[q * d + j] * xs;
            } else {
                // the bucket position of features_kernel, in FP32 (FP64
                // division is slow here, and the value is rounded to FP16)
                const int i = j - d;
                const float g = (float)(HQ[q * m + i] - o[i]);
                float pos = (g + 0.5f) / ((float)span[i] + 1.0f);
                pos = pos < -1.0f ? -1.0f : (pos > 2.0f ? 2.0f : pos);
                v = pos - 0.5f;
            }
        }
        *reinterpret_cast<__half *>(act + tc_off(r, j, K0)) = __float2half_rn(v);
    }
    tc_fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tbase_s;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lanes
    uint32_t phase = 0;

    // D[:, dcol .. dcol + N) = act[128 x K] x W^T.  A thread holds its
    // PER 16-byte pieces of a weight chunk in registers: the next chunk's
    // loads are issued before the wait for the current chunk's MMAs.
    constexpr int PER = TC_MAXN * (TC_KC / 8) / TC_ROWS;
    auto layer = [&](int K, const __half *__restrict__ W, int N, uint32_t dcol) {
        const int pieces = N * (TC_KC / 8);
        uint4 reg[PER];
        auto fetch = [&](int kc) {
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int p = tid + u * TC_ROWS;
                if (p < pieces)
                    reg[u] = *reinterpret_cast<const uint4 *>(W + (int64_t)(p >> 3) * K + kc +
                                                              8 * (p & 7));
            }
        };
        fetch(0);
        for (int kc = 0; kc < K; kc += TC_KC) {
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int p = tid + u * TC_ROWS;
                if (p < pieces) {
                    const int nr = p >> 3, j = p & 7;
                    *reinterpret_cast<uint4 *>(wb + ((nr >> 3) * (TC_KC / 8) + j) * 128 +
                                               (nr & 7) * 16) = reg[u];
                }
            }
            tc_fence_async_smem();
            tc_fence_before();
            __syncthreads();
            const bool go = s_stuck == 0;
            if (tid == 0 && go) {
                tc_fence_after();
                const uint32_t idesc = tc_idesc(TC_ROWS, N);
#pragma unroll
                for (int s2 = 0; s2 < TC_KC / 16; ++s2) {
                    const int kg = kc + 16 * s2;
                    const uint64_t a = tc_desc(act + (kg >> 3) * 128, 128, (uint32_t)K * 16);
                    const uint64_t b = tc_desc(wb + (2 * s2) * 128, 128, (TC_KC / 8) * 128);
                    tc_mma(tbase + dcol, a, b, idesc, (kc | s2) != 0 ? 1u : 0u);
                }
                tc_commit(&bar);
            }
            if (kc + TC_KC < K) fetch(kc + TC_KC);  // in flight while the MMAs run
            if (go) {
                if (!tc_wait(&bar, phase)) s_stuck = 1;
                phase ^= 1;
            }
            tc_fence_after();
        }
    };
    // bias, ReLU, FP16: the next layer's input (K = N columns)
    auto relu_out = [&](uint32_t dcol, const float *__restrict__ bias, int N) {
        for (int n0 = 0; n0 < N; n0 += 16) {
            float v[16];
            tc_ld16(tbase + lane_base + dcol + (uint32_t)n0, v);
            __align__(16) __half hv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) hv[i] = __float2half_rn(fmaxf(v[i] + __ldg(bias + n0 + i), 0.0f));
            *reinterpret_cast<uint4 *>(act + tc_off(tid, n0, N)) = *reinterpret_cast<const uint4 *>(hv);
            *reinterpret_cast<uint4 *>(act + tc_off(tid, n0 + 8, N)) =
                *reinterpret_cast<const uint4 *>(hv + 8);
        }
        tc_fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    };
    layer(K0, W1, H, 0);
    relu_out(0, b1, H);
    layer(H, W2, H, 256);
    relu_out(256, b2, H);
    layer(H, W3, C, 0);
    // logits, softmax, and the row's output
    float z[TC_MAXC];
#pragma unroll
    for (int h2 = 0; h2 < TC_MAXC / 16; ++h2) {
        if (h2 * 16 < C) {
            float v[16];
            tc_ld16(tbase + lane_base + (uint32_t)(h2 * 16), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) z[h2 * 16 + i] = h2 * 16 + i < C ? v[i] + __ldg(b3 + h2 * 16 + i) : -INFINITY;
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) z[h2 * 16 + i] = -INFINITY;
        }
    }
    const int64_t q = r0 + tid;
    const bool stuck = s_stuck != 0;
    if (tid < rows && q < n) {
        float mx = -INFINITY;
#pragma unroll
        for (int c = 0; c < TC_MAXC; ++c) mx = fmaxf(mx, z[c]);
        float sum = 0.0f;
#pragma unroll
        for (int c = 0; c < TC_MAXC; ++c) sum += c < C ? __expf(z[c] - mx) : 0.0f;
        const float inv = 1.0f / sum;
        if (prob) {
#pragma unroll
            for (int c = 0; c < TC_MAXC; ++c)
                if (c < C) prob[q * C + c] = stuck ? NAN : __expf(z[c] - mx) * inv;
        } else {
            float cdf = 0.0f;
            int sl = 0;
            for (int c = 0; c < C - 1; ++c) {
                cdf += __expf(z[c] - mx) * inv;
                if (cdf <= eps) sl = c + 1; else break;
            }
            start[q] = (stuck || sl <= shift) ? 0 : sl - shift;
        }
    }
    if (tid == 0 && stuck && err) atomicOr(err, 16);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
    }
}

}  // namespace

// The tensor-core forward pass takes networks with hidden = 256, classes a
// multiple of 16 up to 32, and n_in a multiple of 64 up to 576 (weights
// 16-byte aligned in the FP16 copy).
static bool tc_eligible(const qw_mlp *mp)
{
    if (mp->H != TC_MAXN || mp->C % 16 != 0 || mp->C > TC_MAXC || mp->n_in % TC_KC != 0 ||
        mp->n_in > TC_MAXK)
        return false;
    const __half *h = mp->p16.as<__half>();
    for (int64_t off : {mp->oW1, mp->oW2, mp->oW3})
        if (reinterpret_cast<uintptr_t>(h + off) % 16 != 0) return false;
    return true;
}

static qw_status launch_mlp_tc(qw_mlp *mp, const float *X, const float *Q, const int32_t *HQ,
                               int64_t n, const IndexView *ix, float xs, float *prob, float eps,
                               int shift, int32_t *start, int *err, cudaStream_t s)
{
    if (n == 0) return QW_OK;
    const int K0 = mp->n_in, Ka = std::max(K0, mp->H);
    // at least 120 KiB, so one CTA per SM: each holds all 512 TMEM columns
    const size_t smem = std::max<size_t>((size_t)TC_ROWS * Ka * 2 + (size_t)TC_MAXN * TC_KC * 2,
                                         (size_t)120 << 10);
    QW_CUDA_TRY(cudaFuncSetAttribute(mlp_forward_tc_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const __half *h = mp->p16.as<__half>();
    const float *p = mp->p32.as<float>();
    // rows per CTA: enough CTAs for every SM (one CTA per SM), 16 to 128
    int dev = 0, sms = 152;
    QW_CUDA_TRY(cudaGetDevice(&dev));
    QW_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t rows = (n + sms - 1) / sms;
    rows = std::min<int64_t>(TC_ROWS, std::max<int64_t>(16, (rows + 15) / 16 * 16));
    mlp_forward_tc_kernel<<<(unsigned)((n + rows - 1) / rows), TC_ROWS, smem, s>>>(
        X, Q, HQ, (int)n, (int)rows, ix ? ix->d : 0, ix ? ix->m : 0, ix ? ix->o : nullptr,
        ix ? ix->span : nullptr, xs, K0, h + mp->oW1, p + mp->ob1, h + mp->oW2, p + mp->ob2,
        h + mp->oW3, p + mp->ob3, mp->H, mp->C, prob, eps, shift, start, err);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_start_model(qw_mlp *mp, const float *Q, const int32_t *HQ, int nq,
                             const IndexView &ix, float xs, float eps, int shift, int32_t *start,
                             cudaStream_t s)
{
    if (nq == 0) return QW_OK;
    if (tc_eligible(mp))
        return launch_mlp_tc(mp, nullptr, Q, HQ, nq, &ix, xs, nullptr, eps, shift, start, nullptr,
                             s);
    const int H = mp->H, C = mp->C, nin = mp->n_in;
    if (mp->t_version != mp->version) {
        QW_TRY(mp->p16t.ensure((size_t)(mp->oW3 + (int64_t)C * H) * sizeof(__half)));
        const __half *h = mp->p16.as<__half>();
        __half *t = mp->p16t.as<__half>();
        transpose_half_kernel<<<152, 256, 0, s>>>(h + mp->oW1, H, nin, t + mp->oW1);
        transpose_half_kernel<<<152, 256, 0, s>>>(h + mp->oW2, H, H, t + mp->oW2);
        transpose_half_kernel<<<152, 256, 0, s>>>(h + mp->oW3, C, H, t + mp->oW3);
        QW_CUDA_TRY(cudaGetLastError());
        mp->t_version = mp->version;
    }
    const size_t smem = (size_t)SM_RB * ((size_t)nin + 2 * (size_t)H + (size_t)C) * sizeof(float);
    QW_CUDA_TRY(cudaFuncSetAttribute(start_model_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const __half *t = mp->p16t.as<__half>();
    const float *p = mp->p32.as<float>();
    start_model_kernel<<<(nq + SM_RB - 1) / SM_RB, SM_THREADS, smem, s>>>(
        Q, HQ, nq, ix.d, ix.m, ix.o, ix.span, xs, t + mp->oW1, p + mp->ob1, t + mp->oW2,
        p + mp->ob2, t + mp->oW3, p + mp->ob3, H, C, eps, shift, start);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status mlp_predict_dev(qw_mlp *mp, const float *X, int64_t n, float *prob, cudaStream_t s)
{
    return qw_mlp_predict(mp, X, n, prob, s);
}

qw_status launch_features(const float *Q, const int32_t *HQ, int64_t nq, const IndexView &ix,
                          float xs, float *F, cudaStream_t s)
{
    if (nq == 0) return QW_OK;
    features_kernel<<<(unsigned)nq, 128, 0, s>>>(Q, HQ, nq, ix.d, ix.m, ix.o, ix.span, xs, F);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_start_levels(const float *prob, int n, int C, float eps, int32_t *start,
                              cudaStream_t s)
{
    if (n == 0) return QW_OK;
    start_level_kernel<<<(n + 127) / 128, 128, 0, s>>>(prob, n, C, eps, start);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status data_rms(const float *X, int64_t count, double *dev_acc, double *out, cudaStream_t s)
{
    QW_CUDA_TRY(cudaMemsetAsync(dev_acc, 0, sizeof(double), s));
    sumsq_kernel<<<152 * 4, 256, 0, s>>>(X, count, dev_acc);
    QW_CUDA_TRY(cudaGetLastError());
    double h = 0.0;
    QW_CUDA_TRY(cudaMemcpyAsync(&h, dev_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    *out = count > 0 ? sqrt(h / (double)count) : 1.0;
    return QW_OK;
}

}  // namespace qw

extern "C" qw_status qw_mlp_predict_tc(qw_mlp *mp, const float *X, int64_t n, float *prob, void *stream)
{
    clear_error();
    if (!mp || !X || !prob) return mlp_error("null pointer");
    if (n < 0 || n > INT32_MAX) return mlp_error("n out of range");
    if (!tc_eligible(mp))
        return mlp_error("qw_mlp_predict_tc: needs hidden = 256, classes a multiple of 16 up to "
                         "32 and n_in a multiple of 64 up to 576");
    cudaStream_t s = (cudaStream_t)stream;
    QW_TRY(mp->tc_err.ensure(sizeof(int)));
    QW_CUDA_TRY(cudaMemsetAsync(mp->tc_err.p, 0, sizeof(int), s));
    QW_TRY(launch_mlp_tc(mp, X, nullptr, nullptr, n, nullptr, 1.0f, prob, 0.0f, 0, nullptr,
                         mp->tc_err.as<int>(), s));
    int h_err = 0;
    QW_CUDA_TRY(cudaMemcpyAsync(&h_err, mp->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err & 16) {
        set_error("qw_mlp_predict_tc: a tensor-core wait gave up");
        return QW_ERR_TIMEOUT;
    }
    return QW_OK;
}
