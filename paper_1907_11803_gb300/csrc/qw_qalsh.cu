// qw_qalsh.cu -- QALSH's query-aware buckets (Section 2; the base method of
// the paper's experiments, Section 6).
//
// The hash function of projection i is the projection itself, p_i(v) = a_i . v
// (no offset, no floor).  At level radius R the bucket of projection i is the
// interval of width w R centred on the query's projection: an object collides
// with the query on projection i when |p_i(o) - p_i(q)| <= w R / 2.  Counting,
// the threshold l, the k + v bound, truncation and top-k are those of the
// bucketed family; the radius rule becomes "every interval holds all the data".
//
// Exactness.  Whether an object lies in an interval is decided on FP64
// projections summed in coordinate order (each product of two floats is exact
// in FP64, so an FMA chain gives the same sums as a multiply-then-add chain),
// with the difference p_i(o) - p_i(q) rounded once and compared with w R / 2.
// That difference is non-decreasing in p_i(o), so the objects inside an
// interval are one contiguous run of a projection's sorted values: two binary
// searches per interval end, evaluated with the same comparison.
//
// Layout (per projection i, tile t; the bucketed family's lid layout):
//   lid[i * nT * kTile + t * kTile + p]  in-tile ids in ascending p_i order
//   qkey[same index]                     the FP64 projection of that id
//   qmin[i], qmax[i]                     smallest and largest p_i over the data
#include "qw_internal.cuh"

#include <algorithm>
#include <climits>

namespace qw {
namespace {

// ---------------------------------------------------------------- FP64 projection
constexpr int PJ_THREADS = 256;
constexpr int PJ_ROWS = 64;     // rows of V per CTA
constexpr int PJ_K = 64;        // coordinates per shared-memory chunk
constexpr int PJ_PER = (QW_MAX_M + 3) / 4;  // projections per thread (4 thread rows)

// out[r * ld_r + i * ld_i] = sum_{j = 0 .. d-1} A[i][j] * V[r][j] in FP64, j ascending.
__global__ void __launch_bounds__(PJ_THREADS) fp64_project_kernel(
    const float *__restrict__ V, int64_t nv, int d, const float *__restrict__ A, int m,
    double *__restrict__ out, int64_t ld_r, int64_t ld_i)
{
    __shared__ float Vs[PJ_ROWS][PJ_K + 1];
    __shared__ float As[QW_MAX_M][PJ_K + 1];
    const int64_t r0 = (int64_t)blockIdx.x * PJ_ROWS;
    const int r = threadIdx.x % PJ_ROWS;       // this thread's row
    const int i0 = threadIdx.x / PJ_ROWS;      // its projections i0, i0 + 4, ...
    double acc[PJ_PER];
#pragma unroll
    for (int p = 0; p < PJ_PER; ++p) acc[p] = 0.0;
    for (int j0 = 0; j0 < d; j0 += PJ_K) {
        const int kc = min(PJ_K, d - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < PJ_ROWS * PJ_K; e += PJ_THREADS) {
            const int rr = e / PJ_K, jj = e % PJ_K;
            const int64_t row = r0 + rr;
            Vs[rr][jj] = (row < nv && jj < kc) ? V[row * d + j0 + jj] : 0.0f;
        }
        for (int e = threadIdx.x; e < m * PJ_K; e += PJ_THREADS) {
            const int ii = e / PJ_K, jj = e % PJ_K;
            As[ii][jj] = jj < kc ? A[(int64_t)ii * d + j0 + jj] : 0.0f;
        }
        __syncthreads();
        for (int jj = 0; jj < kc; ++jj) {
            const double x = (double)Vs[r][jj];
#pragma unroll
            for (int p = 0; p < PJ_PER; ++p) {
                const int i = i0 + 4 * p;
                if (i < m) acc[p] = fma((double)As[i][jj], x, acc[p]);
            }
        }
    }
    const int64_t row = r0 + r;
    if (row >= nv) return;
#pragma unroll
    for (int p = 0; p < PJ_PER; ++p) {
        const int i = i0 + 4 * p;
        if (i < m) out[row * ld_r + (int64_t)i * ld_i] = acc[p];
    }
}

// ---------------------------------------------------------------- order-preserving keys
// Unsigned 64-bit key with the order of the double (finite values; -0 < +0).
__device__ __forceinline__ unsigned long long dkey(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double dval(unsigned long long k)
{
    const unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Smallest and largest projection of every projection i (P: m rows of ldp).
__global__ void key_minmax_kernel(const double *__restrict__ P, int64_t n, int64_t ldp,
                                  unsigned long long *kmin, unsigned long long *kmax)
{
    const int i = blockIdx.y;
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = dkey(P[(int64_t)i * ldp + j]);
        lo = min(lo, k);
        hi = max(hi, k);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(kmin + i, lo);
        atomicMax(kmax + i, hi);
    }
}

__global__ void key_to_double_kernel(const unsigned long long *k, int n, double *out, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = dval(k[i]);
    out[i] = v;
    if (!isfinite(v)) atomicOr(err, 2);  // a projection is not finite
}

// ---------------------------------------------------------------- per-tile sort
constexpr int QS_THREADS = 1024;
constexpr int QS_HALF = kTile / 2;           // entries sorted at once in shared memory
constexpr int QS_OUT = kTile / QS_THREADS;   // merged outputs per thread

// Ascending by (key, in-tile id): a strict total order (ids are distinct).
__device__ __forceinline__ bool key_less(unsigned long long ka, uint16_t la,
                                         unsigned long long kb, uint16_t lb)
{
    return ka < kb || (ka == kb && la < lb);
}

// One CTA orders one (tile, projection) pair: each half of the tile (up to
// 16,384 entries, 10 bytes each) is bitonic-sorted in shared memory and
// written back over its own projections in P (as keys), then the two sorted
// halves are merged (merge-path split, 32 outputs per thread) into qkey / lid.
__global__ void __launch_bounds__(QS_THREADS) qalsh_sort_kernel(
    double *P, int64_t n, int nT, uint16_t *__restrict__ tlid,
    double *__restrict__ qkey, uint16_t *__restrict__ lid)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem);
    uint16_t *sl = reinterpret_cast<uint16_t *>(sk + QS_HALF);
    const int t = blockIdx.x;
    const int i = blockIdx.y;
    const int64_t base = (int64_t)t * kTile;
    const int len = (int)min((int64_t)kTile, n - base);
    const int64_t seg = (int64_t)i * nT * kTile + base;
    unsigned long long *gk = reinterpret_cast<unsigned long long *>(P) + seg;
    const int nh = len > QS_HALF ? 2 : 1;
    for (int h = 0; h < nh; ++h) {
        const int hb = h * QS_HALF;
        const int hl = min(QS_HALF, len - hb);
        int Pn = 1;
        while (Pn < hl) Pn <<= 1;
        for (int j = threadIdx.x; j < Pn; j += QS_THREADS) {
            if (j < hl) {
                sk[j] = dkey(P[seg + hb + j]);
                sl[j] = (uint16_t)(hb + j);
            } else {
                sk[j] = ~0ull;  // after every finite projection
                sl[j] = 0xffff;
            }
        }
        __syncthreads();
        for (int k = 2; k <= Pn; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int x = threadIdx.x; x < (Pn >> 1); x += QS_THREADS) {
                    const int a = 2 * x - (x & (jj - 1));
                    const int c = a + jj;
                    const bool up = (a & k) == 0;
                    if (key_less(sk[c], sl[c], sk[a], sl[a]) == up) {
                        const unsigned long long tk = sk[a]; sk[a] = sk[c]; sk[c] = tk;
                        const uint16_t tl = sl[a]; sl[a] = sl[c]; sl[c] = tl;
                    }
                }
                __syncthreads();
            }
        }
        if (nh == 1) {
            for (int j = threadIdx.x; j < hl; j += QS_THREADS) {
                qkey[seg + j] = dval(sk[j]);
                lid[seg + j] = sl[j];
            }
        } else {
            for (int j = threadIdx.x; j < hl; j += QS_THREADS) {
                gk[hb + j] = sk[j];
                tlid[seg + hb + j] = sl[j];
            }
        }
        __syncthreads();
    }
    if (nh == 1) return;
    // merge the sorted halves [0, QS_HALF) and [QS_HALF, len) of the segment
    const unsigned long long *ka = gk, *kb = gk + QS_HALF;
    const uint16_t *la = tlid + seg, *lb = tlid + seg + QS_HALF;
    const int nA = QS_HALF, nB = len - QS_HALF;
    const int o0 = threadIdx.x * QS_OUT;
    if (o0 >= len) return;
    int lo = max(0, o0 - nB), hi = min(o0, nA);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_less(kb[o0 - mid - 1], lb[o0 - mid - 1], ka[mid], la[mid])) hi = mid;
        else lo = mid + 1;
    }
    int ia = lo, ib = o0 - lo;
    const int o1 = min(len, o0 + QS_OUT);
    for (int o = o0; o < o1; ++o) {
        const bool takeA = ia < nA && (ib >= nB || key_less(ka[ia], la[ia], kb[ib], lb[ib]));
        if (takeA) {
            qkey[seg + o] = dval(ka[ia]);
            lid[seg + o] = la[ia];
            ++ia;
        } else {
            qkey[seg + o] = dval(kb[ib]);
            lid[seg + o] = lb[ib];
            ++ib;
        }
    }
}

// ---------------------------------------------------------------- per-query setup
// The query's projections are in st.g (as FP64 bits).  top: one below the
// first radius R = c^j at which every projection's interval holds the whole
// data, so that the level loop's "R > top" is the radius rule.
__global__ void qalsh_setup_kernel(int nb, int m, const double *__restrict__ qmin,
                                   const double *__restrict__ qmax, double half_unit, int cgrow,
                                   QueryState st, int *err)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    int64_t topR = 1;
    for (int i = 0; i < m; ++i) {
        const double pq = __longlong_as_double((long long)st.g[(int64_t)q * m + i]);
        int64_t R = 1;
        for (;;) {
            const double h = __dmul_rn(half_unit, (double)R);
            if (fabs(__dsub_rn(qmin[i], pq)) <= h && fabs(__dsub_rn(qmax[i], pq)) <= h) break;
            if (R > INT64_MAX / cgrow) {
                atomicOr(err, 2);  // no radius of int64 reaches every object
                break;
            }
            R *= cgrow;
        }
        topR = max(topR, R);
    }
    const int64_t top = topR - 1;
    st.top[q] = top;
    st.active[q] = 1;
    st.ncand[q] = 0;
    st.nprev[q] = 0;
    st.cross[q] = 0;
    st.term[q] = 0;
    st.levels[q] = 0;
    st.finalR[q] = 0;
    st.scan_level[q] = 0;
    st.scan_last[q] = 0;
    st.scan_full[q] = 0;
    st.nkeep[q] = 0;
    st.start[q] = 0;
    st.fb[q] = 0;
    atomicMax(st.max_top, (unsigned long long)top);
}

}  // namespace

qw_status launch_fp64_project(const float *V, int64_t nv, int d, const float *A, int m,
                              double *out, int64_t ld_r, int64_t ld_i, cudaStream_t s)
{
    if (nv == 0) return QW_OK;
    const int64_t blocks = (nv + PJ_ROWS - 1) / PJ_ROWS;
    fp64_project_kernel<<<(unsigned)blocks, PJ_THREADS, 0, s>>>(V, nv, d, A, m, out, ld_r, ld_i);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_qalsh_extent(const double *P, int64_t n, int64_t ldp, int m,
                              unsigned long long *kscratch, double *qmin, double *qmax, int *err,
                              cudaStream_t s)
{
    QW_CUDA_TRY(cudaMemsetAsync(kscratch, 0xff, (size_t)m * 8, s));
    QW_CUDA_TRY(cudaMemsetAsync(kscratch + m, 0, (size_t)m * 8, s));
    const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    key_minmax_kernel<<<dim3(gx, (unsigned)m), 256, 0, s>>>(P, n, ldp, kscratch, kscratch + m);
    QW_CUDA_TRY(cudaGetLastError());
    key_to_double_kernel<<<(m + 127) / 128, 128, 0, s>>>(kscratch, m, qmin, err);
    QW_CUDA_TRY(cudaGetLastError());
    key_to_double_kernel<<<(m + 127) / 128, 128, 0, s>>>(kscratch + m, m, qmax, err);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_qalsh_sort(double *P, int64_t n, int m, int nT, uint16_t *tlid, double *qkey,
                            uint16_t *lid, cudaStream_t s)
{
    const size_t smem = (size_t)QS_HALF * (sizeof(unsigned long long) + sizeof(uint16_t));
    QW_CUDA_TRY(cudaFuncSetAttribute(qalsh_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    qalsh_sort_kernel<<<dim3((unsigned)nT, (unsigned)m), QS_THREADS, smem, s>>>(P, n, nT, tlid,
                                                                             qkey, lid);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_qalsh_setup(const IndexView &ix, int nb, QueryState &st, int cgrow, int *err,
                             cudaStream_t s)
{
    QW_CUDA_TRY(cudaMemsetAsync(st.max_top, 0, sizeof(unsigned long long), s));
    if (nb == 0) return QW_OK;
    qalsh_setup_kernel<<<(nb + 127) / 128, 128, 0, s>>>(nb, ix.m, ix.qmin, ix.qmax, ix.qhalf,
                                                        cgrow, st, err);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
