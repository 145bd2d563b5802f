// qw_noalloc.cu -- qw_run_workload_noalloc: the level-synchronous query path
// for callers that cannot allocate device memory at query time.
//
// All working memory of a call lives in one file-scope device array of
// QW_STATIC_SCRATCH_BYTES; the call carves it into the per-batch query state,
// counters, candidate profiles and candidate lists, and answers the queries in
// batches that fit.  It calls no cudaMalloc / cudaFree and nothing that
// allocates.  The kernels are the ones qw_run_workload launches.
#include "qw_internal.cuh"

#include <algorithm>
#include <string>

namespace qw {
namespace {

// The scratch array.  In host code this name is a host-side stand-in, not a
// device address: host code passes the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_qw_static_scratch[QW_STATIC_SCRATCH_BYTES];

// Device address of the scratch array on the current device, looked up with
// that device current at every call: the lookup is cheap, and an address
// cached across calls would outlive a cudaDeviceReset that reloads the module.
// The first lookup on a device loads the library's module there.
qw_status scratch_address(unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_qw_static_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static scratch)");
    if (!p) {
        set_error("qw_run_workload_noalloc: static scratch has no device address");
        return QW_ERR_CUDA;
    }
    *out = reinterpret_cast<unsigned char *>(p);
    return QW_OK;
}

// The index's arrays must be on the current device, where the scratch is.
qw_status index_on_current_device(const IndexView &ix)
{
    int dev = -1;
    QW_CUDA_TRY(cudaGetDevice(&dev));
    cudaPointerAttributes attr{};
    QW_CUDA_TRY(cudaPointerGetAttributes(&attr, ix.X));
    if (attr.type != cudaMemoryTypeDevice || attr.device != dev) {
        set_error("qw_run_workload_noalloc: the index lives on another device than the current "
                  "one; make its device current");
        return QW_ERR_ARG;
    }
    return QW_OK;
}

constexpr size_t kAlign = 256;

size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Bytes of scratch a batch of B queries needs (every block 256-byte aligned).
size_t batch_bytes(size_t B, int m, int nT, int cap)
{
    size_t total = kAlign;                           // error word + largest anchored id
    total += up(B * m * sizeof(int32_t));            // query bucket ids
    total += up(B * m * sizeof(int64_t));            // anchored query ids
    total += 5 * up(B * sizeof(int64_t));            // top, finalR, scan_level, scan_last, scan_full
    total += 9 * up(B * sizeof(int32_t));            // active, ncand, nprev, cross, term, levels,
                                                     // nkeep, start, fb
    total += up(B * (size_t)nT * kTile);             // collision counters
    total += up(B * (size_t)nT * kHistBins * 4);     // per-tile candidate profiles
    total += up(B * (size_t)nT * 3 * 4);             // per-tile emit plan
    total += up(B * 2 * 4);                          // per-query plan
    total += 2 * up(B * (size_t)cap * 4);            // candidate ids and counts
    return total;
}

qw_status noalloc_arg_error(const char *msg)
{
    set_error(std::string("qw_run_workload_noalloc: ") + msg);
    return QW_ERR_ARG;
}

}  // namespace
}  // namespace qw

using namespace qw;

extern "C" qw_status qw_run_workload_noalloc(qw_index *index, const float *queries, int64_t nq,
                                             int32_t k, int64_t *ids, float *dists,
                                             int64_t *stats, void *stream)
{
    clear_error();
    IndexParams P;
    if (!index || index_params(index, &P) != QW_OK) return noalloc_arg_error("index is null");
    const IndexView &ix = P.view;
    if (nq < 0) return noalloc_arg_error("nq < 0");
    if (nq > 0 && (!queries || !ids || !dists)) return noalloc_arg_error("null pointer");
    if (k < 1 || (int64_t)k > ix.n) return noalloc_arg_error("k must be in [1, n]");
    if ((int64_t)k + P.v > QW_MAX_CAND) return noalloc_arg_error("k + v exceeds 4096");
    if (nq == 0) return QW_OK;
    const int m = ix.m, d = ix.d, nT = ix.nT;
    const int cap = k + P.v;

    // largest batch that fits the static array
    size_t B = 0;
    {
        const size_t one = batch_bytes(1, m, nT, cap);
        if (one > QW_STATIC_SCRATCH_BYTES) {
            return noalloc_arg_error(
                ("one query needs " + std::to_string(one) + " bytes of working memory; the static "
                 "scratch holds " + std::to_string((size_t)QW_STATIC_SCRATCH_BYTES) +
                 " (index too large for this entry point)").c_str());
        }
        B = QW_STATIC_SCRATCH_BYTES / one;
        while (B > 1 && batch_bytes(B, m, nT, cap) > QW_STATIC_SCRATCH_BYTES) --B;
        B = std::min<size_t>(B, (size_t)std::min<int64_t>(nq, 65535));
    }
    QW_TRY(index_on_current_device(ix));
    unsigned char *base = nullptr;
    QW_TRY(scratch_address(&base));

    // carve the scratch
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + off;
        off += up(bytes);
        return p;
    };
    unsigned char *hdr = take(kAlign);
    int *err = reinterpret_cast<int *>(hdr);
    QueryState st;
    st.max_top = reinterpret_cast<unsigned long long *>(hdr + 8);
    st.fb_count = reinterpret_cast<unsigned long long *>(hdr + 16);
    int32_t *hq = reinterpret_cast<int32_t *>(take(B * m * sizeof(int32_t)));
    st.g = reinterpret_cast<int64_t *>(take(B * m * sizeof(int64_t)));
    st.top = reinterpret_cast<int64_t *>(take(B * 8));
    st.finalR = reinterpret_cast<int64_t *>(take(B * 8));
    st.scan_level = reinterpret_cast<int64_t *>(take(B * 8));
    st.scan_last = reinterpret_cast<int64_t *>(take(B * 8));
    st.scan_full = reinterpret_cast<int64_t *>(take(B * 8));
    st.active = reinterpret_cast<int32_t *>(take(B * 4));
    st.ncand = reinterpret_cast<int32_t *>(take(B * 4));
    st.nprev = reinterpret_cast<int32_t *>(take(B * 4));
    st.cross = reinterpret_cast<int32_t *>(take(B * 4));
    st.term = reinterpret_cast<int32_t *>(take(B * 4));
    st.levels = reinterpret_cast<int32_t *>(take(B * 4));
    st.nkeep = reinterpret_cast<int32_t *>(take(B * 4));
    st.start = reinterpret_cast<int32_t *>(take(B * 4));
    st.fb = reinterpret_cast<int32_t *>(take(B * 4));
    st.counters = reinterpret_cast<uint32_t *>(take(B * (size_t)nT * kTile));
    st.tile_hist = reinterpret_cast<int32_t *>(take(B * (size_t)nT * kHistBins * 4));
    st.tile_plan = reinterpret_cast<int32_t *>(take(B * (size_t)nT * 3 * 4));
    st.qplan = reinterpret_cast<int32_t *>(take(B * 2 * 4));
    st.cand = reinterpret_cast<int32_t *>(take(B * (size_t)cap * 4));
    st.cand_col = reinterpret_cast<int32_t *>(take(B * (size_t)cap * 4));
    if (off > QW_STATIC_SCRATCH_BYTES) {
        set_error("qw_run_workload_noalloc: internal scratch layout overflow");
        return QW_ERR_CUDA;
    }

    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t b0 = 0; b0 < nq; b0 += (int64_t)B) {
        const int nb = (int)std::min<int64_t>((int64_t)B, nq - b0);
        const float *Qb = queries + b0 * d;
        // the error word and the largest anchored id start at zero every batch
        QW_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
        if (ix.qkey) {
            // QALSH index: FP64 projections into st.g, then the radius rule
            QW_TRY(launch_fp64_project(Qb, nb, d, P.A, m, reinterpret_cast<double *>(st.g), m, 1,
                                       s));
            QW_TRY(launch_qalsh_setup(ix, nb, st, P.c, err, s));
        } else {
            QW_TRY(launch_hash(Qb, nb, d, P.A, P.b, m, P.w, hq, m, 1, err, nullptr, s));
            QW_TRY(launch_query_setup(ix, hq, nb, st, s));
        }
        unsigned long long max_top = 0;
        int h_err = 0;
        QW_CUDA_TRY(cudaMemcpyAsync(&max_top, st.max_top, sizeof(max_top), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_err & 2) {
            set_error(ix.qkey ? "qw_run_workload_noalloc: no radius below 2^63 makes a query's "
                                "intervals hold the whole data"
                              : "qw_run_workload_noalloc: a query bucket id falls outside int32");
            return QW_ERR_RANGE;
        }
        int64_t R = 1, Rp = 1;
        for (int level = 0;; ++level) {
            QW_TRY(launch_level(ix, nb, level, R, Rp, P.l, P.c, st, s));
            QW_TRY(launch_decide(nb, level, R, cap, st, s));
            if ((unsigned long long)R > max_top) break;
            if (level > 62) {
                set_error("qw_run_workload_noalloc: level limit reached");
                return QW_ERR_TIMEOUT;
            }
            Rp = R;
            R *= P.c;
        }
        QW_TRY(launch_collect(ix, nb, P.l, cap, st, stats ? stats + b0 * QW_NSTAT : nullptr, s));
        QW_TRY(launch_rerank(ix, Qb, nb, k, cap, st, ids + b0 * k, dists + b0 * k, s));
    }
    return QW_OK;
}
