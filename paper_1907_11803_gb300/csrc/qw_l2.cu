// qw_l2.cu -- the workload cache split of Section 4 on the GPU's L2.
//
// The paper divides a cache C into an index part C_I and a data part C_D and
// picks size(C_I) to minimise the IO of the whole workload (Eq. 4).  On
// GB300 the cache is the 126 MB L2.  Part of it can be set aside for
// persisting lines (cudaLimitPersistingL2CacheSize), and an access-policy
// window attached to a launch marks a fraction (the hit ratio) of one address
// range as persisting: those lines stay in the set-aside while the rest of
// the traffic streams through the normal part.  Here the set-aside S is
// divided into
//   - an index window, attached to the collision-counting launches, over the
//     index structure every (query, tile, level) pass reads first: the bucket
//     summaries (bitmap path) or the sorted id arrays (level path);
//   - a data window, attached to the rerank launch, over the rows the
//     candidates are read from (the locality-ordered copy on the bitmap path).
// A window of W bytes whose share is S_X gets hit ratio min(1, S_X / W).
// qw_l2_split_model restates Eq. 4 for this cache; the autotuner and the
// benchmark sweep the split on the paper's grid (its QALSH_Opt setting).
//
// Windows change which lines stay in L2, never what a kernel computes.
#include "qw_l2.cuh"

#include <math.h>

#include <algorithm>

namespace qw {

namespace {

struct DeviceL2 {
    bool known = false;
    size_t max_setaside = 0;  // cudaDevAttrMaxPersistingL2CacheSize
    size_t max_window = 0;    // cudaDevAttrMaxAccessPolicyWindowSize
};

constexpr int kMaxDevices = 64;
DeviceL2 g_dev[kMaxDevices];

double region_traffic(double U, double A, double S)
{
    if (U <= 0.0) return 0.0;
    const double rereads = A > U ? A - U : 0.0;
    const double kept = S >= U ? 1.0 : S / U;
    return U + rereads * (1.0 - kept);
}

}  // namespace

int32_t l2_split_model(double S, double UI, double AI, double UD, double AD)
{
    const double v[5] = {S, UI, AI, UD, AD};
    for (double x : v)
        if (!(x >= 0.0) || !isfinite(x)) return -1;
    if (!(S > 0.0)) return -1;
    int best = 0;
    double best_cost = 0.0;
    for (int p = 0; p <= 1000; ++p) {
        const double SI = S * (double)p / 1000.0;
        const double cost = region_traffic(UI, AI, SI) + region_traffic(UD, AD, S - SI);
        if (p == 0 || cost < best_cost) {
            best = p;
            best_cost = cost;
        }
    }
    return best;
}

void l2_release(L2Owner *o)
{
    if (!o || !o->raised) return;
    bool failed = cudaCtxResetPersistingL2Cache() != cudaSuccess;
    failed |= cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, o->old_limit) != cudaSuccess;
    if (failed) (void)cudaGetLastError();
    o->raised = false;
}

qw_status L2Session::begin(L2Owner *owner, int mode, int permille, const L2Region &index,
                           const L2Region &data, cudaStream_t s)
{
    on = false;
    setaside = 0;
    index_permille = 0;
    if (mode == QW_L2_OFF || s == nullptr) return QW_OK;
    int dev = 0;
    QW_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return QW_OK;
    DeviceL2 &dl = g_dev[dev];
    if (!dl.known) {
        int a = 0, b = 0;
        QW_CUDA_TRY(cudaDeviceGetAttribute(&a, cudaDevAttrMaxPersistingL2CacheSize, dev));
        QW_CUDA_TRY(cudaDeviceGetAttribute(&b, cudaDevAttrMaxAccessPolicyWindowSize, dev));
        dl.max_setaside = a > 0 ? (size_t)a : 0;
        dl.max_window = b > 0 ? (size_t)b : 0;
        dl.known = true;
    }
    if (dl.max_setaside == 0 || dl.max_window == 0) return QW_OK;
    if (!owner->raised) {
        // raising the set-aside is costly (about 0.4 ms per change, measured);
        // it stays raised for the index's lifetime
        size_t old = 0;
        QW_CUDA_TRY(cudaDeviceGetLimit(&old, cudaLimitPersistingL2CacheSize));
        if (old < dl.max_setaside) {
            if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, dl.max_setaside) !=
                cudaSuccess) {
                (void)cudaGetLastError();  // no set-aside here (MIG, MPS): no windows
                return QW_OK;
            }
            owner->raised = true;
            owner->old_limit = old;
        }
    }
    size_t got = 0;
    QW_CUDA_TRY(cudaDeviceGetLimit(&got, cudaLimitPersistingL2CacheSize));
    if (got == 0) return QW_OK;
    cudaStreamAttrValue old{};
    QW_CUDA_TRY(cudaStreamGetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &old));
    old_window = old.accessPolicyWindow;
    stream = s;
    on = true;
    setaside = got;
    if (mode == QW_L2_MODEL) {
        const double UI = (double)std::min(index.bytes, dl.max_window);
        const double UD = (double)std::min(data.bytes, dl.max_window);
        const int32_t p = l2_split_model((double)got, UI, index.reads, UD, data.reads);
        index_permille = p < 0 ? 500 : p;
    } else {
        index_permille = std::min(1000, std::max(0, permille));
    }
    const double SI = (double)got * index_permille / 1000.0;
    make_window(index, SI, dl.max_window, &win_index);
    make_window(data, (double)got - SI, dl.max_window, &win_data);
    return QW_OK;
}

void L2Session::make_window(const L2Region &r, double share, size_t max_window,
                            cudaAccessPolicyWindow *w)
{
    *w = cudaAccessPolicyWindow{};
    const size_t bytes = std::min(r.bytes, max_window);
    if (!r.base || bytes == 0 || share <= 0.0) return;  // num_bytes 0: no window
    w->base_ptr = const_cast<void *>(r.base);
    w->num_bytes = bytes;
    w->hitRatio = (float)std::min(1.0, share / (double)bytes);
    w->hitProp = cudaAccessPropertyPersisting;
    w->missProp = cudaAccessPropertyNormal;  // the rest of the window: plain LRU lines
}

qw_status L2Session::use(L2Use which, cudaStream_t s)
{
    if (!on) return QW_OK;
    cudaStreamAttrValue v{};
    if (which == L2Use::Index) v.accessPolicyWindow = win_index;
    if (which == L2Use::Data) v.accessPolicyWindow = win_data;
    QW_CUDA_TRY(cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &v));
    return QW_OK;
}

cudaAccessPolicyWindow L2Session::window(L2Use which) const
{
    if (!on) return cudaAccessPolicyWindow{};
    return which == L2Use::Index ? win_index
                                 : which == L2Use::Data ? win_data : cudaAccessPolicyWindow{};
}

void L2Session::end()
{
    // best effort on every return path; a failure here leaves no error
    // pending for the caller's next CUDA call
    if (on && stream) {
        cudaStreamAttrValue v{};
        v.accessPolicyWindow = old_window;
        if (cudaStreamSetAttribute(stream, cudaStreamAttributeAccessPolicyWindow, &v) !=
            cudaSuccess)
            (void)cudaGetLastError();
    }
    on = false;
    stream = nullptr;
}

}  // namespace qw

extern "C" int32_t qw_l2_split_model(double setaside, double index_bytes, double index_reads,
                                     double data_bytes, double data_reads)
{
    return qw::l2_split_model(setaside, index_bytes, index_reads, data_bytes, data_reads);
}

// ---- read bandwidth of a buffer of a given size (a measuring tool)
//
// Every thread reads 16-byte words of the buffer in a grid-stride loop with
// loads cached in L2 only (ld.global.cg), so a buffer smaller than L2 measures
// what L2 delivers to the SMs and a buffer much larger than L2 measures HBM.
// The XOR of what was read goes to a sink so the loads are not removed.
namespace {

__global__ void __launch_bounds__(256) read_probe_kernel(const uint4 *__restrict__ p, int64_t n16,
                                                         int passes, unsigned int *sink)
{
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every thread reads the same elements on every pass: after the first
    // pass they are L2 hits when the buffer fits L2 (loads bypass L1)
    for (int pass = 0; pass < passes; ++pass) {
        int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(p + i), b = __ldcg(p + i + stride);
            const uint4 c = __ldcg(p + i + 2 * stride), d = __ldcg(p + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^
                   d.y ^ d.z ^ d.w ^ (uint32_t)pass;
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(p + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    acc = __reduce_xor_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0 && acc == 0x9e3779b9u) atomicAdd(sink, 1u);
}

}  // namespace

extern "C" qw_status qw_measure_read_bandwidth(int64_t bytes, int32_t reps, double *gbs,
                                               void *stream)
{
    using namespace qw;
    clear_error();
    if (bytes < 16 || reps < 1 || !gbs) {
        set_error("qw_measure_read_bandwidth: bytes >= 16, reps >= 1, gbs non-null");
        return QW_ERR_ARG;
    }
    const int64_t n16 = bytes / 16;
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf buf, sink;
    QW_TRY(buf.ensure((size_t)n16 * 16));
    QW_TRY(sink.ensure(16));
    QW_CUDA_TRY(cudaMemsetAsync(buf.p, 0x5a, (size_t)n16 * 16, s));
    QW_CUDA_TRY(cudaMemsetAsync(sink.p, 0, 16, s));
    int dev = 0, n_sm = 0;
    QW_CUDA_TRY(cudaGetDevice(&dev));
    QW_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = n_sm * 8;
    cudaEvent_t e0, e1;
    QW_CUDA_TRY(cudaEventCreate(&e0));
    QW_CUDA_TRY(cudaEventCreate(&e1));
    double best = 0.0;
    // one untimed launch brings a small buffer into L2 (and the clocks up);
    // each timed launch reads the buffer `passes` times (about 2 GB in all), so
    // the launch itself costs little against a small buffer
    const int passes = (int)std::max<int64_t>(
        1, std::min<int64_t>(4096, ((int64_t)2 << 30) / (n16 * 16)));
    for (int w = 0; w < 3; ++w)
        read_probe_kernel<<<grid, 256, 0, s>>>(buf.as<uint4>(), n16, passes,
                                               sink.as<unsigned int>());
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        read_probe_kernel<<<grid, 256, 0, s>>>(buf.as<uint4>(), n16, passes,
                                               sink.as<unsigned int>());
        cudaEventRecord(e1, s);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_status(e, "qw_measure_read_bandwidth");
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.0f) best = fmax(best, (double)passes * n16 * 16.0 / (ms * 1e-3) / 1e9);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    QW_CUDA_TRY(cudaGetLastError());
    *gbs = best;
    return QW_OK;
}
