// qw_api.cu -- the C ABI (include/qwlsh.h): argument checks, device memory
// of the index and its workspace, and the order of kernel launches.  No step
// of the method's arithmetic runs on the host.
#include "qw_internal.cuh"
#include "qw_l2.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

namespace qw {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

qw_status cuda_status(cudaError_t e, const char *what)
{
    std::string msg = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    set_error(msg);
    return e == cudaErrorMemoryAllocation ? QW_ERR_OOM : QW_ERR_CUDA;
}

qw_status DevBuf::ensure(size_t want)
{
    if (want <= bytes) return QW_OK;
    release();
    if (want == 0) return QW_OK;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        (void)cudaGetLastError();
        set_error("device allocation of " + std::to_string(want) + " bytes failed");
        return QW_ERR_OOM;
    }
    bytes = want;
    return QW_OK;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

// Pinned host memory the GPU reads directly (on GB300: Grace memory over
// NVLink-C2C).  The pointer is valid on host and device (unified addressing).
struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
    HostBuf() = default;
    HostBuf(const HostBuf &) = delete;
    HostBuf &operator=(const HostBuf &) = delete;
    ~HostBuf() { release(); }
    qw_status ensure(size_t want)
    {
        if (want <= bytes) return QW_OK;
        release();
        void *h = nullptr;
        cudaError_t e = cudaHostAlloc(&h, want, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("pinned host allocation of " + std::to_string(want) + " bytes failed");
            return QW_ERR_OOM;
        }
        void *dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, h, 0);
        if (e != cudaSuccess || dp != h) {
            (void)cudaGetLastError();
            cudaFreeHost(h);
            set_error("pinned host memory is not addressable at the same address on the device");
            return QW_ERR_CUDA;
        }
        p = h;
        bytes = want;
        return QW_OK;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

static qw_status arg_error(const std::string &msg)
{
    set_error(msg);
    return QW_ERR_ARG;
}

}  // namespace qw

using namespace qw;

struct qw_index {
    int64_t n = 0;
    int d = 0, m = 0, c = 2, v = 0, l = 1;
    float w = 1.0f;
    int nT = 0;
    int32_t span_max = 0;
    int64_t n_fixups = 0;
    DevBuf X, A, b, o, span, lid, dir_bid, dir_off, dir_start, dir_cnt, Xb, xnorm, Cg, Xcr;
    bool shadow = false;
    bool bitmaps = false;               // level bitmaps for QW_PATH_BITMAP
    bool host_bitmaps = false;          // ... kept in pinned host memory (bm_host)
    bool proj_tc = false;               // data projected on the tensor cores at build
    int family = QW_FAMILY_E2LSH;       // bucket family (QW_FAMILY_*)
    DevBuf qkey, qmin, qmax;            // QALSH: sorted FP64 projections, their extent
    HostBuf bm_host;
    DevBuf bm, bm_base, bm_nb, bm_lvl, bm_J, bid_prefix, prefix_off, perm, bm_sum, Xloc, inv, hloc;
    int hloc_bytes = 0, hloc_stride = 0;
    int bm_maxJ = 0;
    float xs = 1.0f;                 // 1 / RMS coordinate of the data (start-model features)
    qw_mlp *start_model = nullptr;   // not owned
    float start_eps = 0.02f;
    LevelGraphCache *graphs = nullptr;  // graph mode of the level loop
    bool tuned = false;                 // qw_autotune ran: QW_PATH_AUTO / batch 0 use these
    int32_t tuned_path = QW_PATH_LEVELS;
    int32_t tuned_batch = 0;
    double l2_levels = 4.0;             // levels per batch of the last call (L2 cost model)
    L2Owner l2_owner;                   // the persisting-L2 set-aside this index raised
    // workspace for queries (grow-only)
    DevBuf w_q, w_hq, w_state, w_counters, w_cand, w_out, w_err, w_order, w_qb, w_ob, w_cbits,
        w_clist, w_bmsel, w_ovf, w_bmwork, w_rdstore;
    int64_t device_bytes = 0;
    qw_profile prof{};
    std::vector<cudaEvent_t> event_pool;

    IndexView view() const
    {
        IndexView v;
        v.X = X.as<float>();
        v.n = n;
        v.d = d;
        v.m = m;
        v.nT = nT;
        v.o = o.as<int32_t>();
        v.span = span.as<int32_t>();
        v.lid = lid.as<uint16_t>();
        v.dir_bid = dir_bid.as<int32_t>();
        v.dir_off = dir_off.as<int32_t>();
        v.dir_start = dir_start.as<int64_t>();
        v.dir_cnt = dir_cnt.as<int32_t>();
        v.bm = host_bitmaps ? bm_host.as<uint4>() : bm.as<uint4>();
        v.bm_base = bm_base.as<int64_t>();
        v.bm_nb = bm_nb.as<int32_t>();
        v.bm_lvl = bm_lvl.as<int32_t>();
        v.bm_J = bm_J.as<int32_t>();
        v.bid_prefix = bid_prefix.as<int64_t>();
        v.perm = perm.as<int32_t>();
        v.bm_sum = bm_sum.as<uint32_t>();
        v.Xloc = Xloc.as<float>();
        v.inv = inv.as<int32_t>();
        v.prefix_off = prefix_off.as<int64_t>();
        v.hloc = hloc.p;
        v.hloc_bytes = hloc_bytes;
        v.hloc_stride = hloc_stride;
        if (family == QW_FAMILY_QALSH) {
            v.qkey = qkey.as<double>();
            v.qmin = qmin.as<double>();
            v.qmax = qmax.as<double>();
            v.qhalf = 0.5 * (double)w;
        }
        return v;
    }
};

// Launch accounting and, in profile mode, CUDA-event timing of every launch
// on the call's stream.
struct LaunchTimer {
    qw_index *ix;
    cudaStream_t s;
    bool on;
    size_t next = 0;
    struct Rec {
        int cls, n;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;

    qw_status event(cudaEvent_t *e)
    {
        if (next == ix->event_pool.size()) {
            cudaEvent_t ne;
            QW_CUDA_TRY(cudaEventCreate(&ne));
            ix->event_pool.push_back(ne);
        }
        *e = ix->event_pool[next++];
        return QW_OK;
    }

    template <class F> qw_status run(int cls, int nlaunch, F &&f)
    {
        cudaEvent_t a = nullptr, b = nullptr;
        if (on) {
            QW_TRY(event(&a));
            QW_TRY(event(&b));
            QW_CUDA_TRY(cudaEventRecord(a, s));
        }
        QW_TRY(f());
        ix->prof.launches[cls] += nlaunch;
        if (on) {
            QW_CUDA_TRY(cudaEventRecord(b, s));
            recs.push_back({cls, nlaunch, a, b});
        }
        return QW_OK;
    }

    qw_status finish()
    {
        if (!on) return QW_OK;
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        for (const Rec &r : recs) {
            float ms = 0.0f;
            QW_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
            ix->prof.ms[r.cls] += ms;
            ix->prof.timed_launches[r.cls] += r.n;
        }
        return QW_OK;
    }
};

qw_status qw::index_params(const qw_index *ix, IndexParams *out)
{
    if (!ix || !out) return QW_ERR_ARG;
    out->view = ix->view();
    out->A = ix->A.as<float>();
    out->b = ix->b.as<float>();
    out->w = ix->w;
    out->c = ix->c;
    out->v = ix->v;
    out->l = ix->l;
    return QW_OK;
}

extern "C" {

const char *qw_version(void) { return "qwlsh-gb300 0.1 (sm_103a)"; }

const char *qw_last_error(void) { return g_last_error.c_str(); }

double qw_collision_probability(double r, double w)
{
    if (!(r > 0.0) || !(w > 0.0)) return NAN;
    const double x = w / r;
    // 1 - 2 Phi(-x) - (2 / (sqrt(2 pi) x)) (1 - exp(-x^2 / 2)),  2 Phi(-x) = erfc(x / sqrt 2)
    return 1.0 - erfc(x * 0.70710678118654752440) -
           (0.79788456080286535588 / x) * (1.0 - exp(-0.5 * x * x));
}

double qw_qalsh_collision_probability(double r, double w)
{
    if (!(r > 0.0) || !(w > 0.0)) return NAN;
    // a . (o - q) ~ N(0, r^2): P(|N(0, r^2)| <= w / 2) = erf(w / (2 sqrt(2) r))
    return erf(w / (2.0 * 1.41421356237309504880 * r));
}

// l = ceil(alpha m), alpha the balance point of p1 = P(1) and p2 = P(c)
// (Section 3.1's collision threshold), for the family's probability P.
static int32_t threshold_of(double (*prob)(double, double), int32_t m, float w, int32_t c,
                            int64_t n, int32_t v, float delta)
{
    if (m < 1 || !(w > 0.0f) || c < 2 || n < 1 || v < 0) return -1;
    const double dl = delta > 0.0f ? (double)delta : exp(-1.0);
    if (!(dl < 1.0)) return -1;
    const double p1 = prob(1.0, w);
    const double p2 = prob((double)c, w);
    double beta = (double)v / (double)n;
    if (beta > 1.0) beta = 1.0;
    if (!(beta > 0.0)) return m;  // no false positive allowed: demand every projection
    const double z = sqrt(log(2.0 / beta) / log(1.0 / dl));
    const double alpha = (z * p1 + p2) / (1.0 + z);
    int32_t l = (int32_t)ceil(alpha * (double)m);
    return std::min(m, std::max(1, l));
}

int32_t qw_collision_threshold(int32_t m, float w, int32_t c, int64_t n, int32_t v, float delta)
{
    return threshold_of(qw_collision_probability, m, w, c, n, v, delta);
}

int32_t qw_qalsh_collision_threshold(int32_t m, float w, int32_t c, int64_t n, int32_t v,
                                     float delta)
{
    return threshold_of(qw_qalsh_collision_probability, m, w, c, n, v, delta);
}

static qw_status hash_impl(const float *V, int64_t nv, int32_t d, const float *A, const float *b,
                           int32_t m, float w, int32_t *H, int64_t *n_fixups, void *stream,
                           bool tc)
{
    clear_error();
    if (!V || !A || !b || !H) return arg_error("qw_hash: null pointer");
    if (nv < 0 || d < 1 || m < 1 || !(w > 0.0f)) return arg_error("qw_hash: bad size or width");
    if (tc && m > 128) return arg_error("qw_hash_tc: m must be <= 128");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf scratch;  // err word + fixup counter
    QW_TRY(scratch.ensure(16));
    int *err = scratch.as<int>();
    unsigned long long *fix = reinterpret_cast<unsigned long long *>(scratch.as<char>() + 8);
    QW_CUDA_TRY(cudaMemsetAsync(scratch.p, 0, 16, s));
    qw_status st = launch_hash(V, nv, d, A, b, m, w, H, m, 1, err, fix, s, tc);
    if (st != QW_OK) { scratch.release(); return st; }
    int h_err = 0;
    unsigned long long h_fix = 0;
    cudaError_t e1 = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaMemcpyAsync(&h_fix, fix, sizeof(h_fix), cudaMemcpyDeviceToHost, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    scratch.release();
    if (e1 != cudaSuccess) return cuda_status(e1, "qw_hash copy");
    if (e2 != cudaSuccess) return cuda_status(e2, "qw_hash copy");
    if (e3 != cudaSuccess) return cuda_status(e3, "qw_hash sync");
    if (n_fixups) *n_fixups = (int64_t)h_fix;
    if (h_err & 2) {
        set_error("qw_hash: a bucket id falls outside int32");
        return QW_ERR_RANGE;
    }
    return QW_OK;
}

qw_status qw_hash(const float *V, int64_t nv, int32_t d, const float *A, const float *b,
                  int32_t m, float w, int32_t *H, int64_t *n_fixups, void *stream)
{
    return hash_impl(V, nv, d, A, b, m, w, H, n_fixups, stream, false);
}

qw_status qw_hash_tc(const float *V, int64_t nv, int32_t d, const float *A, const float *b,
                     int32_t m, float w, int32_t *H, int64_t *n_fixups, void *stream)
{
    return hash_impl(V, nv, d, A, b, m, w, H, n_fixups, stream, true);
}

// QALSH index: FP64 projections of the data, per (projection, tile) sorted
// with their in-tile ids; the projections' extent for the radius rule.  No
// bucket ids: anchors and spans are zero.
static qw_status build_qalsh(qw_index *ix, cudaStream_t s)
{
    const int64_t n = ix->n;
    const int d = ix->d, m = ix->m, nT = ix->nT;
    const size_t slots = (size_t)m * nT * kTile;
    DevBuf P, tlid, scratch;
    QW_TRY(P.ensure(slots * sizeof(double)));
    QW_TRY(tlid.ensure(slots * sizeof(uint16_t)));
    QW_TRY(scratch.ensure(16 + (size_t)m * 16));
    int *err = scratch.as<int>();
    QW_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    // row j of projection i at P[i * nT * kTile + j]: each (projection, tile)
    // segment sits where its sorted copy goes
    QW_TRY(launch_fp64_project(ix->X.as<float>(), n, d, ix->A.as<float>(), m, P.as<double>(), 1,
                               (int64_t)nT * kTile, s));
    QW_TRY(ix->qmin.ensure((size_t)m * sizeof(double)));
    QW_TRY(ix->qmax.ensure((size_t)m * sizeof(double)));
    QW_TRY(launch_qalsh_extent(P.as<double>(), n, (int64_t)nT * kTile, m,
                               reinterpret_cast<unsigned long long *>(scratch.as<char>() + 16),
                               ix->qmin.as<double>(), ix->qmax.as<double>(), err, s));
    QW_TRY(ix->lid.ensure(slots * sizeof(uint16_t)));
    QW_TRY(ix->qkey.ensure(slots * sizeof(double)));
    QW_CUDA_TRY(cudaMemsetAsync(ix->lid.p, 0, ix->lid.bytes, s));
    QW_CUDA_TRY(cudaMemsetAsync(ix->qkey.p, 0, ix->qkey.bytes, s));
    QW_TRY(launch_qalsh_sort(P.as<double>(), n, m, nT, tlid.as<uint16_t>(), ix->qkey.as<double>(),
                             ix->lid.as<uint16_t>(), s));
    QW_TRY(ix->o.ensure((size_t)m * sizeof(int32_t)));
    QW_TRY(ix->span.ensure((size_t)m * sizeof(int32_t)));
    QW_CUDA_TRY(cudaMemsetAsync(ix->o.p, 0, ix->o.bytes, s));
    QW_CUDA_TRY(cudaMemsetAsync(ix->span.p, 0, ix->span.bytes, s));
    ix->span_max = 0;
    int h_err = 0;
    QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err & 2) {
        set_error("qw_build_index: a data projection is not finite");
        return QW_ERR_RANGE;
    }
    {
        DevBuf acc;
        QW_TRY(acc.ensure(16));
        double rms = 1.0;
        QW_TRY(data_rms(ix->X.as<float>(), n * (int64_t)d, acc.as<double>(), &rms, s));
        ix->xs = rms > 0.0 ? (float)(1.0 / rms) : 1.0f;
    }
    if (ix->shadow) {
        QW_TRY(ix->Xb.ensure((size_t)n * d * 2));
        QW_TRY(ix->xnorm.ensure((size_t)n * sizeof(float)));
        QW_TRY(ix->Cg.ensure((size_t)((n + 127) / 128) * d * 2));
        QW_TRY(ix->Xcr.ensure((size_t)n * sizeof(float2)));
        QW_TRY(launch_shadow_bf16(ix->X.as<float>(), n, d, ix->Xb.p, ix->xnorm.as<float>(),
                                  ix->Cg.p, s, ix->Xcr.as<float2>()));
    }
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    ix->device_bytes = (int64_t)(ix->X.bytes + ix->A.bytes + ix->b.bytes + ix->o.bytes +
                                 ix->span.bytes + ix->lid.bytes + ix->qkey.bytes +
                                 ix->qmin.bytes + ix->qmax.bytes + ix->Xb.bytes +
                                 ix->xnorm.bytes + ix->Cg.bytes + ix->Xcr.bytes);
    return QW_OK;
}

static qw_status build_impl(qw_index *ix, const float *data, const float *A, const float *b,
                            int32_t mem, int32_t ab_mem, cudaStream_t s)
{
    const int64_t n = ix->n;
    const int d = ix->d, m = ix->m;
    const cudaMemcpyKind kind = mem == QW_MEM_HOST ? cudaMemcpyHostToDevice
                                                   : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind ab_kind = ab_mem == QW_MEM_HOST ? cudaMemcpyHostToDevice
                                                         : cudaMemcpyDeviceToDevice;
    QW_TRY(ix->X.ensure((size_t)n * d * sizeof(float)));
    QW_TRY(ix->A.ensure((size_t)m * d * sizeof(float)));
    QW_TRY(ix->b.ensure((size_t)m * sizeof(float)));
    QW_CUDA_TRY(cudaMemcpyAsync(ix->X.p, data, (size_t)n * d * sizeof(float), kind, s));
    QW_CUDA_TRY(cudaMemcpyAsync(ix->A.p, A, (size_t)m * d * sizeof(float), ab_kind, s));
    QW_CUDA_TRY(cudaMemcpyAsync(ix->b.p, b, (size_t)m * sizeof(float), ab_kind, s));
    if (ix->family == QW_FAMILY_QALSH) return build_qalsh(ix, s);

    // 1. bucket ids of the data, projection-major (m x n)
    DevBuf Ht, scratch;
    QW_TRY(Ht.ensure((size_t)n * m * sizeof(int32_t)));
    QW_TRY(scratch.ensure(64));
    int *err = scratch.as<int>();
    unsigned long long *fix = reinterpret_cast<unsigned long long *>(scratch.as<char>() + 8);
    QW_CUDA_TRY(cudaMemsetAsync(scratch.p, 0, 16, s));
    QW_TRY(launch_hash(ix->X.as<float>(), n, d, ix->A.as<float>(), ix->b.as<float>(), m, ix->w,
                       Ht.as<int32_t>(), 1, n, err, fix, s, ix->proj_tc));

    // 2. anchors and spans
    QW_TRY(ix->o.ensure((size_t)m * sizeof(int32_t)));
    QW_TRY(ix->span.ensure((size_t)m * sizeof(int32_t)));
    DevBuf hmax;
    QW_TRY(hmax.ensure((size_t)m * sizeof(int32_t)));
    {
        std::vector<int32_t> init_lo(m, INT32_MAX), init_hi(m, INT32_MIN);
        QW_CUDA_TRY(cudaMemcpyAsync(ix->o.p, init_lo.data(), m * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
        QW_CUDA_TRY(cudaMemcpyAsync(hmax.p, init_hi.data(), m * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
        QW_TRY(launch_minmax(Ht.as<int32_t>(), n, m, ix->o.as<int32_t>(), hmax.as<int32_t>(), s));
    }
    std::vector<int32_t> h_o(m), h_hi(m);
    int h_err = 0;
    unsigned long long h_fix = 0;
    QW_CUDA_TRY(cudaMemcpyAsync(h_o.data(), ix->o.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaMemcpyAsync(h_hi.data(), hmax.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaMemcpyAsync(&h_fix, fix, sizeof(h_fix), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err & 2) {
        set_error("qw_build_index: a data bucket id falls outside int32");
        return QW_ERR_RANGE;
    }
    ix->n_fixups = (int64_t)h_fix;
    std::vector<int32_t> h_span(m);
    ix->span_max = 0;
    for (int i = 0; i < m; ++i) {
        int64_t sp = (int64_t)h_hi[i] - (int64_t)h_o[i];
        if (sp > 2147483646LL) {
            set_error("qw_build_index: bucket span of a projection exceeds int32");
            return QW_ERR_RANGE;
        }
        h_span[i] = (int32_t)sp;
        ix->span_max = std::max(ix->span_max, h_span[i]);
    }
    QW_CUDA_TRY(cudaMemcpyAsync(ix->span.p, h_span.data(), m * sizeof(int32_t),
                                cudaMemcpyHostToDevice, s));

    // 3. directory capacity per (projection, tile): min(tile length, span + 1)
    const int nT = ix->nT;
    std::vector<int64_t> h_start((size_t)m * nT);
    int64_t total = 0;
    for (int i = 0; i < m; ++i) {
        for (int t = 0; t < nT; ++t) {
            int64_t len = std::min<int64_t>(kTile, n - (int64_t)t * kTile);
            h_start[(size_t)i * nT + t] = total;
            total += std::min<int64_t>(len, (int64_t)h_span[i] + 1);
        }
    }
    QW_TRY(ix->lid.ensure((size_t)m * nT * kTile * sizeof(uint16_t)));
    QW_CUDA_TRY(cudaMemsetAsync(ix->lid.p, 0, ix->lid.bytes, s));
    QW_TRY(ix->dir_bid.ensure((size_t)total * sizeof(int32_t)));
    QW_TRY(ix->dir_off.ensure((size_t)total * sizeof(int32_t)));
    QW_TRY(ix->dir_start.ensure((size_t)m * nT * sizeof(int64_t)));
    QW_TRY(ix->dir_cnt.ensure((size_t)m * nT * sizeof(int32_t)));
    QW_CUDA_TRY(cudaMemcpyAsync(ix->dir_start.p, h_start.data(), h_start.size() * sizeof(int64_t),
                                cudaMemcpyHostToDevice, s));
    QW_TRY(launch_tile_sort(Ht.as<int32_t>(), n, m, nT, ix->o.as<int32_t>(), ix->lid.as<uint16_t>(),
                            ix->dir_bid.as<int32_t>(), ix->dir_off.as<int32_t>(),
                            ix->dir_start.as<int64_t>(), ix->dir_cnt.as<int32_t>(), s));
    {
        DevBuf acc;
        QW_TRY(acc.ensure(16));
        double rms = 1.0;
        QW_TRY(data_rms(ix->X.as<float>(), n * (int64_t)d, acc.as<double>(), &rms, s));
        ix->xs = rms > 0.0 ? (float)(1.0 / rms) : 1.0f;
    }
    if (ix->bitmaps) {
        BitmapLayout lay;
        QW_TRY(bitmap_layout(h_span, nT, ix->c, &lay));
        if (lay.total > (int64_t)INT32_MAX) {  // bitmaps are numbered in 31 bits
            set_error("qw_build_index: bitmap table too large");
            return QW_ERR_RANGE;
        }
        const size_t bm_bytes = (size_t)lay.total * kBmUint4 * sizeof(uint4);
        if (ix->host_bitmaps)
            QW_TRY(ix->bm_host.ensure(bm_bytes));
        else
            QW_TRY(ix->bm.ensure(bm_bytes));
        QW_TRY(ix->bm_base.ensure((size_t)m * sizeof(int64_t)));
        QW_TRY(ix->bm_nb.ensure((size_t)m * sizeof(int32_t)));
        QW_TRY(ix->bm_lvl.ensure((size_t)m * kBmLevels * sizeof(int32_t)));
        QW_TRY(ix->bm_J.ensure((size_t)m * sizeof(int32_t)));
        if (ix->host_bitmaps)
            memset(ix->bm_host.p, 0, ix->bm_host.bytes);
        else
            QW_CUDA_TRY(cudaMemsetAsync(ix->bm.p, 0, ix->bm.bytes, s));
        QW_CUDA_TRY(cudaMemcpyAsync(ix->bm_base.p, lay.base.data(), m * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, s));
        QW_CUDA_TRY(cudaMemcpyAsync(ix->bm_nb.p, lay.nb.data(), m * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
        QW_CUDA_TRY(cudaMemcpyAsync(ix->bm_lvl.p, lay.lvl.data(), lay.lvl.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
        QW_CUDA_TRY(cudaMemcpyAsync(ix->bm_J.p, lay.J.data(), m * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
        ix->bm_maxJ = *std::max_element(lay.J.begin(), lay.J.end());
        // per projection, objects with bid < b for b = 0 .. span + 1
        std::vector<int64_t> poff(m);
        int64_t ptot = 0;
        for (int i = 0; i < m; ++i) {
            poff[i] = ptot;
            ptot += (int64_t)h_span[i] + 2;
        }
        QW_TRY(ix->bid_prefix.ensure((size_t)ptot * sizeof(int64_t)));
        QW_TRY(ix->prefix_off.ensure((size_t)m * sizeof(int64_t)));
        QW_CUDA_TRY(cudaMemsetAsync(ix->bid_prefix.p, 0, ix->bid_prefix.bytes, s));
        QW_CUDA_TRY(cudaMemcpyAsync(ix->prefix_off.p, poff.data(), m * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, s));
        // internal (locality) order of the bitmaps
        std::vector<int32_t> h_perm;
        {
            std::vector<float> hX, hA;
            try {
                hX.resize((size_t)n * d);
                hA.resize((size_t)m * d);
            } catch (const std::bad_alloc &) {
                set_error("qw_build_index: out of host memory for the locality order");
                return QW_ERR_OOM;
            }
            QW_CUDA_TRY(cudaMemcpyAsync(hX.data(), ix->X.p, hX.size() * sizeof(float),
                                        cudaMemcpyDeviceToHost, s));
            QW_CUDA_TRY(cudaMemcpyAsync(hA.data(), ix->A.p, hA.size() * sizeof(float),
                                        cudaMemcpyDeviceToHost, s));
            QW_CUDA_TRY(cudaStreamSynchronize(s));
            QW_TRY(locality_order(hX.data(), n, d, hA.data(), m, h_perm));
        }
        QW_TRY(ix->perm.ensure((size_t)n * sizeof(int32_t)));
        QW_CUDA_TRY(cudaMemcpyAsync(ix->perm.p, h_perm.data(), (size_t)n * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
        QW_TRY(ix->bm_sum.ensure((size_t)lay.total * (kBmUint4 / 32) * sizeof(uint32_t)));
        QW_TRY(launch_bitmap_build(ix->view(), ix->c, ix->bm_maxJ, Ht.as<int32_t>(),
                                   ix->host_bitmaps ? ix->bm_host.as<uint4>() : ix->bm.as<uint4>(),
                                   ix->bm_sum.as<uint32_t>(), lay.total, s));
        QW_TRY(ix->Xloc.ensure((size_t)n * d * sizeof(float)));
        QW_TRY(ix->inv.ensure((size_t)n * sizeof(int32_t)));
        QW_TRY(launch_locality_copy(ix->X.as<float>(), ix->perm.as<int32_t>(), n, d,
                                    ix->Xloc.as<float>(), ix->inv.as<int32_t>(), s));
        // anchored bucket ids per internal id, in the narrowest width that holds the spans
        const int32_t smax = *std::max_element(h_span.begin(), h_span.end());
        ix->hloc_bytes = smax < 256 ? 1 : (smax < 65536 ? 2 : 4);
        ix->hloc_stride = (m * ix->hloc_bytes + 15) / 16 * 16;
        QW_TRY(ix->hloc.ensure((size_t)n * ix->hloc_stride));
        QW_CUDA_TRY(cudaMemsetAsync(ix->hloc.p, 0, ix->hloc.bytes, s));
        QW_TRY(launch_hloc_build(ix->view(), Ht.as<int32_t>(), ix->hloc.p, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));  // the host order must outlive its upload
        QW_TRY(launch_bid_prefix(ix->view(), ix->bid_prefix.as<int64_t>(),
                                 ix->prefix_off.as<int64_t>(), s));
    }
    if (ix->shadow) {
        // residuals to 128-row group means, in the rows' order of the rerank
        // (the locality-ordered copy when the index has bitmaps)
        QW_TRY(ix->Xb.ensure((size_t)n * d * 2));
        QW_TRY(ix->xnorm.ensure((size_t)n * sizeof(float)));
        QW_TRY(ix->Cg.ensure((size_t)((n + 127) / 128) * d * 2));
        const float *Xs = ix->bitmaps ? ix->Xloc.as<float>() : ix->X.as<float>();
        QW_TRY(ix->Xcr.ensure((size_t)n * sizeof(float2)));
        QW_TRY(launch_shadow_bf16(Xs, n, d, ix->Xb.p, ix->xnorm.as<float>(), ix->Cg.p, s,
                                  ix->Xcr.as<float2>()));
    }
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    ix->device_bytes = (int64_t)(ix->Xb.bytes + ix->xnorm.bytes + ix->Cg.bytes + ix->Xcr.bytes + ix->X.bytes + ix->A.bytes + ix->b.bytes + ix->o.bytes +
                                 ix->span.bytes + ix->lid.bytes + ix->dir_bid.bytes +
                                 ix->dir_off.bytes + ix->dir_start.bytes + ix->dir_cnt.bytes +
                                 ix->bm.bytes + ix->bm_base.bytes + ix->bm_nb.bytes +
                                 ix->bm_lvl.bytes + ix->bm_J.bytes + ix->bid_prefix.bytes +
                                 ix->prefix_off.bytes + ix->perm.bytes + ix->bm_sum.bytes +
                                 ix->Xloc.bytes + ix->inv.bytes + ix->hloc.bytes);
    return QW_OK;
}

qw_status qw_build_index(const float *data, int64_t n, int32_t d, const float *A, const float *b,
                         const qw_index_params *p, int32_t mem, void *stream, qw_index **out)
{
    clear_error();
    if (!out) return arg_error("qw_build_index: out is null");
    *out = nullptr;
    if (!data || !p) return arg_error("qw_build_index: null pointer");
    if ((A == nullptr) != (b == nullptr))
        return arg_error("qw_build_index: give both A and b, or neither (drawn from params->seed)");
    if (mem != QW_MEM_DEVICE && mem != QW_MEM_HOST) return arg_error("qw_build_index: bad mem flag");
    if (n < 1 || n > 2147483647LL) return arg_error("qw_build_index: n must be in [1, 2^31)");
    if (d < 1) return arg_error("qw_build_index: d must be >= 1");
    if (p->m < 1 || p->m > QW_MAX_M) return arg_error("qw_build_index: m must be in [1, 127]");
    if (!(p->w > 0.0f) || !isfinite(p->w)) return arg_error("qw_build_index: w must be > 0");
    if (p->c < 2) return arg_error("qw_build_index: c must be an integer >= 2");
    if (p->v < 0) return arg_error("qw_build_index: v must be >= 0");
    if (p->l < 0 || p->l > p->m) return arg_error("qw_build_index: l must be in [0, m]");
    if (p->host_bitmaps && !p->bitmaps)
        return arg_error("qw_build_index: host_bitmaps needs bitmaps");
    if (p->family != QW_FAMILY_E2LSH && p->family != QW_FAMILY_QALSH)
        return arg_error("qw_build_index: unknown family");
    if (p->family == QW_FAMILY_QALSH && p->bitmaps)
        return arg_error("qw_build_index: QW_FAMILY_QALSH has no level bitmaps");
    if (p->family == QW_FAMILY_QALSH && p->projection != QW_PROJ_FP32)
        return arg_error("qw_build_index: QW_FAMILY_QALSH projects in FP64 (projection must be "
                         "QW_PROJ_FP32)");
    qw_index *ix = new (std::nothrow) qw_index();
    if (!ix) {
        set_error("qw_build_index: host allocation failed");
        return QW_ERR_OOM;
    }
    ix->n = n;
    ix->d = d;
    ix->m = p->m;
    ix->w = p->w;
    ix->c = p->c;
    ix->v = p->v;
    ix->family = p->family;
    ix->l = p->l > 0 ? p->l
                     : (p->family == QW_FAMILY_QALSH
                            ? qw_qalsh_collision_threshold(p->m, p->w, p->c, n, p->v, p->delta)
                            : qw_collision_threshold(p->m, p->w, p->c, n, p->v, p->delta));
    if (ix->l < 1) {
        delete ix;
        return arg_error("qw_build_index: cannot derive the collision threshold (bad delta?)");
    }
    ix->nT = (int)((n + kTile - 1) / kTile);
    ix->shadow = p->shadow_bf16 != 0;
    ix->bitmaps = p->bitmaps != 0;
    ix->host_bitmaps = ix->bitmaps && p->host_bitmaps != 0;
    if (p->projection != QW_PROJ_FP32 && p->projection != QW_PROJ_TENSOR) {
        delete ix;
        return arg_error("qw_build_index: unknown projection");
    }
    if (p->projection == QW_PROJ_TENSOR && p->m > 128) {
        delete ix;
        return arg_error("qw_build_index: QW_PROJ_TENSOR needs m <= 128");
    }
    ix->proj_tc = p->projection == QW_PROJ_TENSOR;
    // no projections given: draw them on the host from the seed (Section 3's
    // a ~ N(0, I_d), b ~ U[0, w); see qw_draw_projections)
    std::vector<float> drawn_A, drawn_b;
    int32_t ab_mem = mem;
    if (!A) {
        drawn_A.resize((size_t)p->m * d);
        drawn_b.resize((size_t)p->m);
        qw_draw_projections(p->seed, p->m, d, p->w, drawn_A.data(), drawn_b.data());
        A = drawn_A.data();
        b = drawn_b.data();
        ab_mem = QW_MEM_HOST;
    }
    qw_status st = build_impl(ix, data, A, b, mem, ab_mem, (cudaStream_t)stream);
    if (st != QW_OK) {
        qw_index_free(ix);
        return st;
    }
    *out = ix;
    return QW_OK;
}

static qw_status run_impl(qw_index *ix, const float *queries, int64_t nq, int k,
                          const qw_query_params *qp, int64_t *ids, float *dists, int64_t *stats,
                          int64_t *cand_ids, int32_t *cand_col, int32_t mem, cudaStream_t s);

// Workspace of one batch on the bitmap path (its default batch size).
constexpr int64_t kBitmapBudget = (int64_t)48 << 30;

// Answer the workload queries listed in `list` (device, n of them) again and
// write their rows of the outputs: on the level path (`rerun` null) for the
// rare queries whose candidates overflow the bitmap path's fixed buffers, or
// with the given settings (the bitmap path from level 0, for queries whose
// learned first level was too late).  The list is copied first: the nested
// call reuses the workspace it lives in.
static qw_status answer_again(qw_index *ix, const float *Qall, const int32_t *HQall,
                              const int32_t *list, int n, int k, int cap, int64_t *f_ids,
                              float *f_dists, int64_t *f_stats, int64_t *f_cids, int32_t *f_ccol,
                              cudaStream_t s, const qw_query_params *rerun = nullptr)
{
    const int d = ix->d, m = ix->m;
    DevBuf lst, q_in, hq_in, o_ids, o_dists, o_stats, o_cids, o_ccol;
    QW_TRY(lst.ensure((size_t)n * sizeof(int32_t)));
    QW_CUDA_TRY(cudaMemcpyAsync(lst.p, list, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                s));
    list = lst.as<int32_t>();
    QW_TRY(q_in.ensure((size_t)n * d * sizeof(float)));
    QW_TRY(hq_in.ensure((size_t)n * m * sizeof(int32_t)));
    QW_TRY(launch_gather(Qall, HQall, list, 0, n, d, m, q_in.as<float>(), hq_in.as<int32_t>(), s));
    if (f_ids) {
        QW_TRY(o_ids.ensure((size_t)n * k * sizeof(int64_t)));
        QW_TRY(o_dists.ensure((size_t)n * k * sizeof(float)));
    }
    if (f_stats) QW_TRY(o_stats.ensure((size_t)n * QW_NSTAT * sizeof(int64_t)));
    if (f_cids) QW_TRY(o_cids.ensure((size_t)n * cap * sizeof(int64_t)));
    if (f_ccol) QW_TRY(o_ccol.ensure((size_t)n * cap * sizeof(int32_t)));
    qw_query_params p{};
    if (rerun) {
        p = *rerun;
    } else {
        // the level path in graph mode, from the learned first levels when a
        // start model is attached (both leave the results unchanged)
        p.path = QW_PATH_LEVELS;
        p.order = QW_ORDER_GIVEN;
        p.graph = 1;
        if (ix->start_model && mlp_inputs(ix->start_model) == ix->d + ix->m)
            p.start = QW_START_LEARNED;
    }
    const qw_profile saved = ix->prof;
    QW_TRY(run_impl(ix, q_in.as<float>(), n, k, &p, o_ids.as<int64_t>(), o_dists.as<float>(),
                    o_stats.as<int64_t>(), o_cids.as<int64_t>(), o_ccol.as<int32_t>(),
                    QW_MEM_DEVICE, s));
    const int64_t nested_fallbacks = ix->prof.bitmap_fallbacks - saved.bitmap_fallbacks;
    ix->prof = saved;
    if (rerun) {
        ix->prof.start_fallbacks += n;
        ix->prof.bitmap_fallbacks += nested_fallbacks;
    } else {
        ix->prof.bitmap_fallbacks += n;
    }
    QW_TRY(launch_scatter(list, 0, n, k, cap, o_ids.as<int64_t>(), o_dists.as<float>(),
                          o_stats.as<int64_t>(), o_cids.as<int64_t>(), o_ccol.as<int32_t>(), f_ids,
                          f_dists, f_stats, f_cids, f_ccol, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));  // the temporaries are freed on return
    return QW_OK;
}

// The level loop of one batch, driven by the host: levels 0..L where c^L
// exceeds the batch's largest useful radius (afterwards every query has
// stopped); with learned starts, a second pass from level 0 for the queries
// that stopped at their learned first level.
static qw_status host_level_loop(qw_index *ix, LaunchTimer &tm, const IndexView &view, int nb,
                                 int cap, bool learned, bool bitmap, int loads, int tpw, int *err,
                                 QueryState &st, cudaStream_t s, int *levels_run)
{
    unsigned long long max_top = 0;
    QW_CUDA_TRY(cudaMemcpyAsync(&max_top, st.max_top, sizeof(max_top), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    for (int pass = 0; pass < 2; ++pass) {
        int64_t R = 1, Rp = 1;
        for (int level = 0;; ++level) {
            if (bitmap && loads != QW_LOADS_TMA) {
                // the bucket numbers apart, so that QW_K_LEVEL times the filter
                // and count passes alone
                QW_TRY(tm.run(QW_K_BUCKET, 1, [&] {
                    return launch_bm_level(view, nb, level, R, Rp, ix->l, ix->c, st, err, loads,
                                           s, nullptr, 1, tpw);
                }));
                const int nl = loads == QW_LOADS_FUSED ? 1 : (st.bm_prof ? 3 : 2);
                QW_TRY(tm.run(QW_K_LEVEL, nl, [&] {
                    return launch_bm_level(view, nb, level, R, Rp, ix->l, ix->c, st, err, loads,
                                           s, nullptr, 2, tpw);
                }));
            } else {
                QW_TRY(tm.run(QW_K_LEVEL, 1, [&] {
                    return bitmap ? launch_bm_level(view, nb, level, R, Rp, ix->l, ix->c, st, err,
                                                    loads, s)
                                  : launch_level(view, nb, level, R, Rp, ix->l, ix->c, st, s);
                }));
            }
            QW_TRY(tm.run(QW_K_DECIDE, 1, [&] {
                ScanStats ss = bitmap ? scan_stats_of(view, ix->c) : ScanStats();
                ss.recount_first = bitmap && learned;
                return launch_decide(nb, level, R, cap, st, s, nullptr, ss);
            }));
            ++*levels_run;
            if ((unsigned long long)R > max_top) break;
            if (level > 62) {
                set_error("qw_run_workload: level limit reached");
                return QW_ERR_TIMEOUT;
            }
            Rp = R;
            R *= ix->c;
        }
        if (!learned) break;
        unsigned long long fbc[2] = {0, 0};
        QW_TRY(tm.run(QW_K_DECIDE, 1, [&] { return launch_fallback(nb, st, s); }));
        QW_CUDA_TRY(cudaMemcpyAsync(fbc, st.fb_count, sizeof(fbc), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        if (pass == 0) {
            ix->prof.start_fallbacks += (int64_t)fbc[0];
            ix->prof.start_levels_skipped += (int64_t)fbc[1];
        }
        if (fbc[0] == 0) break;
        QW_CUDA_TRY(cudaMemsetAsync(st.fb_count, 0, 16, s));
    }
    return QW_OK;
}

// The bitmap path's two-pass work buffers for B queries: byte size, and (when
// st is given) their places in `base`: counters; per item (query, tile) its
// (q, t) and its m bitmap numbers (int32, rows padded to 4 entries); per group
// a work entry and its projection mask; per (parity, item) the live-group
// mask; per (query, projection) the bucket's bitmap number in tile 0.
static size_t bm_work_layout(int64_t B, int nT, int m, QueryState *st, char *base = nullptr)
{
    const size_t items = (size_t)B * nT;
    const size_t mpad = (size_t)(m + 3) / 4 * 4;
    const size_t mw = (size_t)(m + 63) / 64;
    auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };
    size_t off = 16;
    const size_t o_qt = off;    off = up16(off + items * sizeof(int2));
    const size_t o_bi = off;    off = up16(off + items * mpad * sizeof(int32_t));
    const size_t o_work = off;  off = up16(off + items * kBmUint4 * sizeof(int32_t));
    const size_t o_amask = off; off = up16(off + 2 * items * (kBmUint4 / 32) * sizeof(uint32_t));
    const size_t o_wmask = off; off = up16(off + items * kBmUint4 * mw * 8);
    const size_t o_bq = off;    off = up16(off + (size_t)B * m * sizeof(int64_t));
    if (st && base) {
        st->bm_nitems = reinterpret_cast<int32_t *>(base);
        st->bm_nwork = st->bm_nitems + 1;
        st->bm_item_qt = reinterpret_cast<int2 *>(base + o_qt);
        st->bm_item_bi = reinterpret_cast<int32_t *>(base + o_bi);
        st->bm_work = reinterpret_cast<int32_t *>(base + o_work);
        st->bm_amask = reinterpret_cast<uint32_t *>(base + o_amask);
        st->bm_wmask = reinterpret_cast<unsigned long long *>(base + o_wmask);
        st->bm_bq = reinterpret_cast<int64_t *>(base + o_bq);
    }
    return off;
}

static qw_status run_impl(qw_index *ix, const float *queries, int64_t nq, int k,
                          const qw_query_params *qp, int64_t *ids, float *dists,
                          int64_t *stats, int64_t *cand_ids, int32_t *cand_col, int32_t mem,
                          cudaStream_t s)
{
    const bool want_cand = cand_ids != nullptr;
    const bool want_ids = ids != nullptr;
    const int m = ix->m, d = ix->d;
    const int cap = k + ix->v;
    const int64_t wpq_bytes = (int64_t)ix->nT * kTile;  // counter bytes per query
    const int path = qp ? qp->path : QW_PATH_AUTO;
    const bool qalsh = ix->family == QW_FAMILY_QALSH;
    // the workload order groups queries by bucket signature (bucketed family)
    const bool order = !qalsh && (!qp || qp->order != QW_ORDER_GIVEN);
    const bool host = mem == QW_MEM_HOST;
    const bool bf16 = qp && qp->rerank == QW_RERANK_BF16;
    const bool bf16_tc = qp && qp->rerank == QW_RERANK_BF16_TC;
    if (bf16 && !ix->shadow) {
        set_error("qw_run_workload: QW_RERANK_BF16 needs an index built with shadow_bf16");
        return QW_ERR_ARG;
    }
    if (bf16_tc && !ix->shadow) {
        set_error("qw_run_workload: QW_RERANK_BF16_TC needs an index built with shadow_bf16");
        return QW_ERR_ARG;
    }
    int csize = 0, tpc = 0;
    const bool fits = cluster_path_fits(ix->view(), &csize, &tpc);
    if (path == QW_PATH_CLUSTER && !fits) {
        set_error("qw_run_workload: the index has more tiles than the cluster path can hold");
        return QW_ERR_ARG;
    }
    const bool learned = qp && qp->start == QW_START_LEARNED;
    if (learned && !ix->start_model) {
        set_error("qw_run_workload: QW_START_LEARNED needs a start model (qw_index_set_start_model)");
        return QW_ERR_ARG;
    }
    if (learned && path == QW_PATH_CLUSTER) {
        set_error("qw_run_workload: learned start levels run on the level path");
        return QW_ERR_ARG;
    }
    const bool graph = qp && qp->graph != 0;
    if (graph && path == QW_PATH_CLUSTER) {
        set_error("qw_run_workload: graph mode runs the level path");
        return QW_ERR_ARG;
    }
    // QW_PATH_AUTO: the tuned path if the index was tuned, else the level path
    int eff_path = path;
    if (eff_path == QW_PATH_AUTO)
        eff_path = (ix->tuned && !learned && !graph) ? ix->tuned_path : QW_PATH_LEVELS;
    // multi-probe runs on the level path only
    if (qp && qp->probes > 0) eff_path = QW_PATH_LEVELS;
    if (path == QW_PATH_BITMAP && !ix->bitmaps) {
        set_error("qw_run_workload: QW_PATH_BITMAP needs an index built with bitmaps");
        return QW_ERR_ARG;
    }
    if (eff_path == QW_PATH_BITMAP && !ix->bitmaps) eff_path = QW_PATH_LEVELS;
    const bool use_cluster = eff_path == QW_PATH_CLUSTER && fits;
    const bool use_bitmap = eff_path == QW_PATH_BITMAP;
    // bitmaps in host memory are read with plain loads (the TMA variant stages
    // device memory only)
    int loads = qp ? qp->bitmap_loads : QW_LOADS_TMA;
    if (loads == QW_LOADS_TMA && ix->host_bitmaps) loads = QW_LOADS_DIRECT;
    const bool tma_loads = loads == QW_LOADS_TMA;
    const int tpw = qp && qp->tiles_per_warp ? qp->tiles_per_warp : 8;
    const int rr_rows = qp && qp->rerank_rows ? qp->rerank_rows : 4;
    // bitmap path, per query: two levels of (tile) candidate bitmaps and lists
    const int64_t cb_bytes = (int64_t)ix->nT * kBmUint4 * (int64_t)sizeof(uint4) * 2;
    // (per query: two levels of tile candidate counts and candidate lists)
    const int64_t cl_bytes = (int64_t)ix->nT * (int64_t)sizeof(int32_t) * 2 +
                             ((int64_t)kQCap * (int64_t)sizeof(uint64_t) + 4) * 2;
    int64_t B = qp && qp->batch > 0 ? qp->batch : 0;
    if (B == 0 && ix->tuned && ix->tuned_batch > 0 && !use_cluster &&
        (path == QW_PATH_AUTO || path == ix->tuned_path))
        B = ix->tuned_batch;
    if (B == 0) {
        // workspace of one batch: 2 GB of counters on the level path; the
        // bitmap path (about 4.3 MB per query at 1M points) takes up to 48 GB,
        // a sixth of the 280 GB HBM, so most workloads run as one batch
        const int64_t budget = use_bitmap ? kBitmapBudget : (int64_t)2 << 30;
        B = use_cluster ? (int64_t)65535
                        : std::max<int64_t>(1, budget / (use_bitmap ? cb_bytes + cl_bytes
                                                                    : wpq_bytes));
    }
    B = std::min<int64_t>(B, std::max<int64_t>(nq, 1));
    B = std::min<int64_t>(B, 65535);
    // bitmap path: (query, tile) item slots are numbered in 23 bits
    if (use_bitmap) B = std::max<int64_t>(1, std::min<int64_t>(B, ((int64_t)1 << 23) / ix->nT));
    auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };

    // ---- workspace
    QW_TRY(ix->w_err.ensure(128));
    QW_TRY(ix->w_hq.ensure((size_t)nq * m * sizeof(int32_t)));       // bucket ids of all queries
    if (!use_cluster && !use_bitmap) QW_TRY(ix->w_counters.ensure((size_t)B * wpq_bytes));
    if (use_bitmap) {
        QW_TRY(ix->w_cbits.ensure((size_t)B * cb_bytes));
        QW_TRY(ix->w_clist.ensure((size_t)B * cl_bytes + 64));
        // per query: flags, recount mark, tie list; then the list-rebuild
        // slots (count, plans, count histograms)
        QW_TRY(ix->w_bmsel.ensure((size_t)B * (2 + kEqCap) * sizeof(int32_t) + 256 +
                                  (size_t)B * sizeof(RdPlan) +
                                  (size_t)B * 2 * kHistBins * sizeof(int32_t) +
                                  (size_t)B * 2 * QW_MAX_M * sizeof(int64_t)));
        // two-pass level: one slot per (query, tile), one work entry per group
        const size_t items = (size_t)B * ix->nT;
        QW_TRY(ix->w_bmwork.ensure(bm_work_layout(B, ix->nT, m, nullptr)));
        // the overflow rebuild's plane store: one wave of slots
        QW_TRY(ix->w_rdstore.ensure((size_t)std::min<int64_t>(B, bm_reduce_wave(ix->nT)) *
                                    ix->nT * kBmUint4 * 8 * sizeof(uint4)));
        QW_TRY(ix->w_ovf.ensure(((size_t)nq + 1) * 2 * sizeof(int32_t)));
    }
    QW_TRY(ix->w_cand.ensure((size_t)B * cap * 2 * sizeof(int32_t)));
    const size_t plan_ints = (size_t)B * ix->nT * (kHistBins + 3) + (size_t)B * 2;
    const size_t st_bytes = (size_t)B * m * 8 + (size_t)B * 8 * 16 + plan_ints * 4 + 256 +
                            (size_t)B * 4 * 2 + 64 + 16 * ((sizeof(LoopCtl) + 15) / 16);
    QW_TRY(ix->w_state.ensure(st_bytes));
    if (learned && mlp_inputs(ix->start_model) != d + m) {
        set_error("qw_run_workload: the start model's input size is not d + m");
        return QW_ERR_ARG;
    }
    // outputs of the whole workload in device memory (the caller's in device mode)
    const size_t o_ids = want_ids ? (size_t)nq * k * sizeof(int64_t) : 0;
    const size_t o_dists = want_ids ? (size_t)nq * k * sizeof(float) : 0;
    const size_t o_stats = stats ? (size_t)nq * QW_NSTAT * sizeof(int64_t) : 0;
    const size_t o_cids = want_cand ? (size_t)nq * cap * sizeof(int64_t) : 0;
    const size_t o_ccol = (want_cand && cand_col) ? (size_t)nq * cap * sizeof(int32_t) : 0;
    const float *Qall = queries;
    int64_t *f_ids = ids, *f_stats = stats, *f_cids = cand_ids;
    float *f_dists = dists;
    int32_t *f_ccol = cand_col;
    if (host) {
        QW_TRY(ix->w_q.ensure((size_t)nq * d * sizeof(float)));
        QW_TRY(ix->w_out.ensure(up16(o_ids) + up16(o_dists) + up16(o_stats) + up16(o_cids) +
                                up16(o_ccol)));
        char *o = ix->w_out.as<char>();
        f_ids = want_ids ? reinterpret_cast<int64_t *>(o) : nullptr;
        o += up16(o_ids);
        f_dists = want_ids ? reinterpret_cast<float *>(o) : nullptr;
        o += up16(o_dists);
        f_stats = stats ? reinterpret_cast<int64_t *>(o) : nullptr;
        o += up16(o_stats);
        f_cids = want_cand ? reinterpret_cast<int64_t *>(o) : nullptr;
        o += up16(o_cids);
        f_ccol = (want_cand && cand_col) ? reinterpret_cast<int32_t *>(o) : nullptr;
        Qall = ix->w_q.as<float>();
    }
    // per-batch staging when the workload is reordered
    const size_t b_ids = want_ids ? (size_t)B * k * sizeof(int64_t) : 0;
    const size_t b_dists = want_ids ? (size_t)B * k * sizeof(float) : 0;
    const size_t b_stats = stats ? (size_t)B * QW_NSTAT * sizeof(int64_t) : 0;
    const size_t b_cids = want_cand ? (size_t)B * cap * sizeof(int64_t) : 0;
    const size_t b_ccol = (want_cand && cand_col) ? (size_t)B * cap * sizeof(int32_t) : 0;
    if (order) {
        QW_TRY(ix->w_order.ensure(up16((size_t)nq * 4) * 2 + order_hist_ints() * 4));
        QW_TRY(ix->w_qb.ensure(up16((size_t)B * d * sizeof(float)) +
                               up16((size_t)B * m * sizeof(int32_t))));
        QW_TRY(ix->w_ob.ensure(up16(b_ids) + up16(b_dists) + up16(b_stats) + up16(b_cids) +
                               up16(b_ccol) + 16));
    }
    QueryState st;
    st.probes = qp ? qp->probes : 0;
    LoopCtl *ctl = nullptr;
    {
        char *p = ix->w_state.as<char>();
        auto take = [&](size_t bytes) { char *r = p; p += (bytes + 15) / 16 * 16; return r; };
        st.g = reinterpret_cast<int64_t *>(take((size_t)B * m * 8));
        st.top = reinterpret_cast<int64_t *>(take((size_t)B * 8));
        st.finalR = reinterpret_cast<int64_t *>(take((size_t)B * 8));
        st.scan_level = reinterpret_cast<int64_t *>(take((size_t)B * 8));
        st.scan_last = reinterpret_cast<int64_t *>(take((size_t)B * 8));
        st.scan_full = reinterpret_cast<int64_t *>(take((size_t)B * 8));
        st.active = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.ncand = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.nprev = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.cross = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.term = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.levels = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.nkeep = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.max_top = reinterpret_cast<unsigned long long *>(take(8));
        st.tile_hist = reinterpret_cast<int32_t *>(take((size_t)B * ix->nT * kHistBins * 4));
        st.tile_plan = reinterpret_cast<int32_t *>(take((size_t)B * ix->nT * 3 * 4));
        st.qplan = reinterpret_cast<int32_t *>(take((size_t)B * 2 * 4));
        st.start = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.fb = reinterpret_cast<int32_t *>(take((size_t)B * 4));
        st.fb_count = reinterpret_cast<unsigned long long *>(take(16));
        ctl = reinterpret_cast<LoopCtl *>(take(sizeof(LoopCtl)));
        if ((size_t)(p - ix->w_state.as<char>()) > ix->w_state.bytes) {
            set_error("internal: query state workspace too small");
            return QW_ERR_CUDA;
        }
    }
    st.counters = ix->w_counters.as<uint32_t>();
    st.cbits = ix->w_cbits.as<uint4>();
    st.level_passes = nullptr;
    st.cb_par = B * ix->nT * kBmUint4;
    if (use_bitmap) {
        // w_clist: qbuf (2 x B x kQCap), then clist_n (2 x B x nT), then qbuf_n (2 x B)
        st.qb_par = B * (int64_t)kQCap;
        st.qbuf = ix->w_clist.as<uint64_t>();
        st.cln_par = B * ix->nT;
        st.clist_n = reinterpret_cast<int32_t *>(st.qbuf + 2 * st.qb_par);
        st.qbn_par = B;
        st.qbuf_n = st.clist_n + 2 * st.cln_par;
        st.bm_ovf = ix->w_bmsel.as<int32_t>();
        st.recount = st.bm_ovf + B;
        st.eqbuf = st.bm_ovf + 2 * B;
        {
            // control words and plans on 16-byte boundaries
            uintptr_t a = reinterpret_cast<uintptr_t>(st.eqbuf + (size_t)B * kEqCap);
            st.rd_ctl = reinterpret_cast<int32_t *>((a + 15) & ~(uintptr_t)15);
        }
        st.rd_plan = reinterpret_cast<RdPlan *>(st.rd_ctl + 16);
        st.rd_hist = reinterpret_cast<int32_t *>(st.rd_plan + B);
        {
            // int64 bitmap numbers on an 8-byte boundary
            uintptr_t a = reinterpret_cast<uintptr_t>(st.rd_hist + (size_t)B * 2 * kHistBins);
            st.rd_bq = reinterpret_cast<int64_t *>((a + 15) & ~(uintptr_t)15);
        }
        st.rd_store = ix->w_rdstore.as<uint4>();
        const int64_t items = B * (int64_t)ix->nT;
        bm_work_layout(B, ix->nT, m, &st, ix->w_bmwork.as<char>());
        st.bm_item_cap = (int32_t)std::min<int64_t>(items, (int64_t)1 << 23);
        st.bm_work_cap = (int32_t)std::min<int64_t>(items * kBmUint4, INT32_MAX);
    }
    // two counters, then the two lists of queries to answer again
    int32_t *ovf_count = use_bitmap ? ix->w_ovf.as<int32_t>() : nullptr;
    int32_t *ovf_list = use_bitmap ? ovf_count + 2 : nullptr;
    int32_t *late_list = use_bitmap ? ovf_list + nq : nullptr;
    if (use_bitmap) QW_CUDA_TRY(cudaMemsetAsync(ovf_count, 0, 2 * sizeof(int32_t), s));
    st.cand = ix->w_cand.as<int32_t>();
    st.cand_col = st.cand + (size_t)B * cap;
    int *err = ix->w_err.as<int>();
    int *queue = reinterpret_cast<int *>(ix->w_err.as<char>() + 32);
    unsigned long long *rows_ctr = reinterpret_cast<unsigned long long *>(ix->w_err.as<char>() + 40);
    unsigned long long *cand_ctr = reinterpret_cast<unsigned long long *>(ix->w_err.as<char>() + 48);
    const IndexView view = ix->view();
    LaunchTimer tm{ix, s, qp && qp->profile != 0};
    if (tm.on) {
        QW_CUDA_TRY(cudaMemsetAsync(ix->w_err.as<char>() + 40, 0, 48, s));
        st.level_passes = reinterpret_cast<unsigned long long *>(ix->w_err.as<char>() + 56);
        if (use_bitmap)
            st.bm_prof = reinterpret_cast<unsigned long long *>(ix->w_err.as<char>() + 64);
    }

    // ---- persisting-L2 windows (the workload's index / data cache split)
    L2Session l2;
    const int l2_mode = qp ? qp->l2_mode : QW_L2_OFF;
    if (l2_mode != QW_L2_OFF) {
        // expected reads: per (query, level) the summaries of every tile
        // (bitmap path) or the 2-byte ids of the level's bucket ranges (level
        // and cluster paths: about c^(L-1) of the span + 1 bids); per query at
        // most k + v data rows
        const double L = std::max(1.0, ix->l2_levels);
        L2Region ri, rd;
        if (use_bitmap) {
            ri.base = ix->bm_sum.p;
            ri.bytes = ix->bm_sum.bytes;
            ri.reads = (double)nq * L * ix->nT * m * 32.0;
            rd.base = ix->Xloc.p;
        } else {
            ri.base = ix->lid.p;
            ri.bytes = ix->lid.bytes;
            const double frac = std::min(1.0, pow((double)ix->c, L - 1.0) / (ix->span_max + 1.0));
            ri.reads = (double)nq * 2.0 * m * (double)ix->n * frac;
            rd.base = ix->X.p;
        }
        rd.bytes = (size_t)ix->n * d * sizeof(float);
        rd.reads = (double)nq * cap * d * sizeof(float);
        QW_TRY(l2.begin(&ix->l2_owner, l2_mode, qp->l2_index_permille, ri, rd, s));
    } else if (ix->l2_owner.raised) {
        // a call without windows after calls with them: put the set-aside back
        // and demote their persisting lines, so this call sees the plain L2
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        l2_release(&ix->l2_owner);
    }
    int levels_run = 0;

    // ---- the whole workload: copy in (host mode), hash, order
    if (host)
        QW_CUDA_TRY(cudaMemcpyAsync(ix->w_q.p, queries, (size_t)nq * d * sizeof(float),
                                    cudaMemcpyHostToDevice, s));
    int32_t *HQall = ix->w_hq.as<int32_t>();
    QW_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (!qalsh)
        QW_TRY(tm.run(QW_K_PROJECT, 2, [&] {
            return launch_hash(Qall, nq, d, ix->A.as<float>(), ix->b.as<float>(), m, ix->w, HQall,
                               m, 1, err, nullptr, s, qp && qp->projection == QW_PROJ_TENSOR);
        }));
    int32_t *perm = nullptr;
    if (order) {
        char *o = ix->w_order.as<char>();
        perm = reinterpret_cast<int32_t *>(o);
        uint32_t *keys = reinterpret_cast<uint32_t *>(o + up16((size_t)nq * 4));
        int32_t *hist = reinterpret_cast<int32_t *>(o + 2 * up16((size_t)nq * 4));
        QW_TRY(tm.run(QW_K_ORDER, 3, [&] { return launch_order(HQall, nq, view, keys, hist, perm, s); }));
    }
    {
        int h_err = 0;
        QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_err & 2) {
            set_error("qw_run_workload: a query bucket id falls outside int32");
            return QW_ERR_RANGE;
        }
    }

    int64_t n_batches = 0;
    if (graph && !use_cluster) {
        if (!ix->graphs && !(ix->graphs = level_graph_cache_new())) {
            set_error("qw_run_workload: out of host memory");
            return QW_ERR_OOM;
        }
        QW_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(LoopCtl), s));
    }
    for (int64_t b0 = 0; b0 < nq; b0 += B) {
        const int nb = (int)std::min<int64_t>(B, nq - b0);
        ++n_batches;
        const float *Qb;
        const int32_t *HQb;
        int64_t *ids_b = nullptr, *stats_b = nullptr, *cids_b = nullptr;
        float *dists_b = nullptr;
        int32_t *ccol_b = nullptr;
        if (order) {
            float *qb = ix->w_qb.as<float>();
            int32_t *hqb = reinterpret_cast<int32_t *>(ix->w_qb.as<char>() +
                                                       up16((size_t)B * d * sizeof(float)));
            QW_TRY(tm.run(QW_K_ORDER, 1, [&] {
                return launch_gather(Qall, HQall, perm, b0, nb, d, m, qb, hqb, s);
            }));
            Qb = qb;
            HQb = hqb;
            char *o = ix->w_ob.as<char>();
            if (want_ids) ids_b = reinterpret_cast<int64_t *>(o);
            o += up16(b_ids);
            if (want_ids) dists_b = reinterpret_cast<float *>(o);
            o += up16(b_dists);
            if (stats) stats_b = reinterpret_cast<int64_t *>(o);
            o += up16(b_stats);
            if (want_cand) cids_b = reinterpret_cast<int64_t *>(o);
            o += up16(b_cids);
            if (want_cand && cand_col) ccol_b = reinterpret_cast<int32_t *>(o);
        } else {
            Qb = Qall + b0 * d;
            HQb = HQall + b0 * m;
            if (want_ids) {
                ids_b = f_ids + b0 * k;
                dists_b = f_dists + b0 * k;
            }
            if (stats) stats_b = f_stats + b0 * QW_NSTAT;
            if (want_cand) cids_b = f_cids + b0 * cap;
            if (want_cand && cand_col) ccol_b = f_ccol + b0 * cap;
        }
        QW_TRY(l2.use(L2Use::Index, s));
        if (use_cluster) {
            int used = 0;
            QW_CUDA_TRY(cudaMemsetAsync(st.nkeep, 0, (size_t)nb * sizeof(int32_t), s));
            QW_TRY(tm.run(QW_K_CLUSTER, 1, [&] {
                return launch_cluster_query(view, HQb, nb, ix->l, ix->c, cap, csize, tpc,
                                            qp ? qp->clusters : 0, st, queue, stats_b, err, s,
                                            &used);
            }));
            int h_err = 0;
            QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            QW_CUDA_TRY(cudaStreamSynchronize(s));
            if (h_err & 4) {
                set_error("qw_run_workload: a staged-copy wait in the cluster kernel gave up");
                return QW_ERR_TIMEOUT;
            }
        } else {
            if (qalsh) {
                // the batch's FP64 projections go to st.g, then the radius rule
                QW_TRY(tm.run(QW_K_PROJECT, 1, [&] {
                    return launch_fp64_project(Qb, nb, d, ix->A.as<float>(), m,
                                               reinterpret_cast<double *>(st.g), m, 1, s);
                }));
                QW_TRY(tm.run(QW_K_SETUP, 1, [&] {
                    return launch_qalsh_setup(view, nb, st, ix->c, err, s);
                }));
                int h_err = 0;
                QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
                QW_CUDA_TRY(cudaStreamSynchronize(s));
                if (h_err & 2) {
                    set_error("qw_run_workload: no radius below 2^63 makes a query's intervals "
                              "hold the whole data");
                    return QW_ERR_RANGE;
                }
            } else {
                QW_TRY(tm.run(QW_K_SETUP, 1, [&] { return launch_query_setup(view, HQb, nb, st, s); }));
            }
            if (learned) {
                QW_TRY(tm.run(QW_K_START, 1, [&] {
                    // bitmap path: start at the predicted last level (its previous
                    // level is recounted); level path: one level before it
                    return launch_start_model(ix->start_model, Qb, HQb, nb, view, ix->xs,
                                              ix->start_eps, use_bitmap ? 0 : 1, st.start, s);
                }));
                QW_TRY(tm.run(QW_K_START, 1, [&] { return launch_clamp_start(nb, st, ix->c, s); }));
                QW_CUDA_TRY(cudaMemsetAsync(st.fb_count, 0, 16, s));
            }
            if (graph) {
                QW_TRY(tm.run(QW_K_LEVEL, 0, [&] {
                    return run_level_graph(ix->graphs, view, nb, ix->l, ix->c, cap, learned,
                                           use_bitmap, loads, tpw, st, ctl, err, s,
                                           l2.window(L2Use::Index));
                }));
            } else {
                QW_TRY(host_level_loop(ix, tm, view, nb, cap, learned, use_bitmap, loads, tpw, err,
                                       st, s, &levels_run));
            }
            QW_TRY(tm.run(QW_K_SELECT, use_bitmap ? (learned ? 4 : 2) : 2, [&] {
                if (use_bitmap)
                    QW_TRY(launch_bm_reduce(view, nb, ix->l, cap, ix->c, st, tma_loads,
                                            (int)std::min<int64_t>(B, bm_reduce_wave(ix->nT)), s));
                if (use_bitmap && learned)
                    QW_TRY(launch_bm_recount(view, nb, ix->l, cap, ix->c, st, s));
                return use_bitmap ? launch_bm_collect(view, nb, ix->l, cap, st, stats_b, want_cand, s)
                                  : launch_collect(view, nb, ix->l, cap, st, stats_b, s);
            }));
            if (use_bitmap)
                QW_TRY(launch_bm_overflow_list(st, nb, order ? perm : nullptr, b0, ovf_list,
                                               late_list, ovf_count, s));
            if (use_bitmap && tm.on) {
                int32_t h_rd = 0;
                QW_CUDA_TRY(cudaMemcpyAsync(&h_rd, st.rd_ctl, sizeof(h_rd), cudaMemcpyDeviceToHost, s));
                QW_CUDA_TRY(cudaStreamSynchronize(s));
                ix->prof.bitmap_overflows += h_rd;
            }
        }
        if (want_cand)
            QW_TRY(tm.run(QW_K_SELECT, 1, [&] { return launch_candidates_out(st, nb, cap, cids_b, ccol_b, s); }));
        if (want_ids) QW_TRY(l2.use(L2Use::Data, s));
        if (want_ids && bf16)
            QW_TRY(tm.run(QW_K_RERANK, 1, [&] {
                return launch_rerank_bf16(view, ix->Xb.p, ix->xnorm.as<float>(),
                                          ix->Xcr.as<float2>(), ix->Cg.p, Qb, nb, k, cap, st,
                                          ids_b, dists_b, tm.on ? rows_ctr : nullptr, s, rr_rows);
            }));
        else if (want_ids && bf16_tc)
            QW_TRY(tm.run(QW_K_RERANK, 1, [&] {
                return launch_rerank_tc(view, ix->Xb.p, ix->xnorm.as<float>(),
                                        ix->Xcr.as<float2>(), ix->Cg.p, Qb, nb, k, cap, st,
                                        ids_b, dists_b, tm.on ? rows_ctr : nullptr, err, s);
            }));
        else if (want_ids)
            QW_TRY(tm.run(QW_K_RERANK, 1, [&] {
                // bitmap path: candidate rows from the locality-ordered copy
                return use_bitmap ? launch_rerank(view, Qb, nb, k, cap, st, ids_b, dists_b, s,
                                                  ix->Xloc.as<float>(), ix->inv.as<int32_t>(),
                                                  rr_rows)
                                  : launch_rerank(view, Qb, nb, k, cap, st, ids_b, dists_b, s,
                                                  nullptr, nullptr, rr_rows);
            }));
        if (want_ids && tm.on)
            QW_TRY(launch_sum_i32(st.nkeep, nb, cand_ctr, s));
        if (order) {
            QW_TRY(tm.run(QW_K_ORDER, 1, [&] {
                return launch_scatter(perm, b0, nb, k, cap, ids_b, dists_b, stats_b, cids_b, ccol_b,
                                      f_ids, f_dists, f_stats, f_cids, f_ccol, s);
            }));
        }
    }
    if (want_ids && bf16_tc) {
        // a tensor-core wait of the pre-filter that gave up (bounded waits; the
        // answers are still exact, every candidate having gone to the exact stages)
        int h_err = 0;
        QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_err & 32) {
            set_error("qw_run_workload: a tensor-core wait in the BF16 pre-filter gave up");
            return QW_ERR_TIMEOUT;
        }
    }
    if (use_bitmap && !graph) {
        // a staged-copy wait of the bitmap kernel that gave up (bounded waits)
        int h_err = 0;
        QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_err & 4) {
            set_error("qw_run_workload: a staged-copy wait in the bitmap kernel gave up");
            return QW_ERR_TIMEOUT;
        }
    }
    if (graph && !use_cluster) {
        // the device-driven loops: their launch counts, the level-limit flag and
        // the learned-start counters, once per call
        LoopCtl h_ctl;
        int h_err = 0;
        QW_CUDA_TRY(cudaMemcpyAsync(&h_ctl, ctl, sizeof(h_ctl), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_err & 8) {
            set_error("qw_run_workload: level limit reached");
            return QW_ERR_TIMEOUT;
        }
        if (h_err & 4) {
            set_error("qw_run_workload: a staged-copy wait in the bitmap kernel gave up");
            return QW_ERR_TIMEOUT;
        }
        // per level: the bucket numbers, filter and count (bitmap path, direct
        // loads), else one counting launch
        ix->prof.launches[QW_K_LEVEL] +=
            (int64_t)h_ctl.iters *
            (use_bitmap && loads == QW_LOADS_DIRECT ? 3 : (use_bitmap && loads == QW_LOADS_FUSED ? 2 : 1));
        levels_run = (int)h_ctl.iters;
        ix->prof.launches[QW_K_DECIDE] += 2 * (int64_t)h_ctl.iters + n_batches * (learned ? 3 : 1);
        if (learned) {
            ix->prof.start_fallbacks += (int64_t)h_ctl.fb_total;
            ix->prof.start_levels_skipped += (int64_t)h_ctl.skipped_total;
        }
    }
    if (use_bitmap) {
        // queries whose candidate lists overflowed the bitmap path's buffers:
        // answered again by the level path; queries whose learned first level
        // was too late: answered again by the bitmap path from level 0 (same
        // results by construction either way); after every read of this
        // call's flags and loop state, which the nested calls reuse
        int32_t n_ovf[2] = {0, 0};
        QW_CUDA_TRY(cudaMemcpyAsync(n_ovf, ovf_count, sizeof(n_ovf), cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        if (n_ovf[0] > 0)
            QW_TRY(answer_again(ix, Qall, HQall, ovf_list, n_ovf[0], k, cap, f_ids, f_dists,
                                f_stats, f_cids, f_ccol, s));
        if (n_ovf[1] > 0) {
            qw_query_params p{};
            p.path = QW_PATH_BITMAP;
            p.order = QW_ORDER_GIVEN;
            p.start = QW_START_PLAIN;
            p.graph = graph ? 1 : 0;
            p.bitmap_loads = loads;
            p.tiles_per_warp = qp ? qp->tiles_per_warp : 0;
            p.rerank_rows = qp ? qp->rerank_rows : 0;
            QW_TRY(answer_again(ix, Qall, HQall, late_list, n_ovf[1], k, cap, f_ids, f_dists,
                                f_stats, f_cids, f_ccol, s, &p));
        }
    }
    if (host) {
        if (want_ids) {
            QW_CUDA_TRY(cudaMemcpyAsync(ids, f_ids, o_ids, cudaMemcpyDeviceToHost, s));
            QW_CUDA_TRY(cudaMemcpyAsync(dists, f_dists, o_dists, cudaMemcpyDeviceToHost, s));
        }
        if (stats) QW_CUDA_TRY(cudaMemcpyAsync(stats, f_stats, o_stats, cudaMemcpyDeviceToHost, s));
        if (want_cand) {
            QW_CUDA_TRY(cudaMemcpyAsync(cand_ids, f_cids, o_cids, cudaMemcpyDeviceToHost, s));
            if (cand_col)
                QW_CUDA_TRY(cudaMemcpyAsync(cand_col, f_ccol, o_ccol, cudaMemcpyDeviceToHost, s));
        }
        QW_CUDA_TRY(cudaStreamSynchronize(s));
    }
    QW_TRY(tm.finish());
    if (tm.on) {
        unsigned long long ctr[6] = {0, 0, 0, 0, 0, 0};
        QW_CUDA_TRY(cudaMemcpy(ctr, ix->w_err.as<char>() + 40, sizeof(ctr), cudaMemcpyDeviceToHost));
        ix->prof.rerank_fp32_rows += (int64_t)((bf16 || bf16_tc) ? ctr[0] : ctr[1]);
        ix->prof.rerank_candidates += (int64_t)ctr[1];
        ix->prof.level_passes += (int64_t)ctr[2];
        ix->prof.bitmap_live_items += (int64_t)ctr[3];
        ix->prof.bitmap_live_groups += (int64_t)ctr[4];
        ix->prof.bitmap_live_words += (int64_t)ctr[5];
    }
    ix->prof.queries += nq;
    if (n_batches > 0 && levels_run > 0 && !use_cluster)
        ix->l2_levels = (double)levels_run / (double)n_batches;
    if (l2_mode != QW_L2_OFF) {
        ix->prof.l2_setaside_bytes = (int64_t)l2.setaside;
        ix->prof.l2_index_permille = l2.on ? l2.index_permille : 0;
    }
    return QW_OK;
}

static qw_status check_workload_args(const qw_index *ix, const float *queries, int64_t nq,
                                     int32_t k, const qw_query_params *qp, int32_t mem)
{
    if (!ix) return arg_error("qw_run_workload: index is null");
    if (nq < 0) return arg_error("qw_run_workload: nq < 0");
    if (nq > 0 && !queries) return arg_error("qw_run_workload: null pointer");
    if (mem != QW_MEM_DEVICE && mem != QW_MEM_HOST) return arg_error("qw_run_workload: bad mem flag");
    if (k < 1 || (int64_t)k > ix->n) return arg_error("qw_run_workload: k must be in [1, n]");
    if ((int64_t)k + ix->v > QW_MAX_CAND) return arg_error("qw_run_workload: k + v exceeds 4096");
    if (qp) {
        if (qp->batch < 0) return arg_error("qw_run_workload: batch < 0");
        if (qp->path < QW_PATH_AUTO || qp->path > QW_PATH_BITMAP)
            return arg_error("qw_run_workload: unknown path");
        if (qp->clusters < 0) return arg_error("qw_run_workload: clusters < 0");
        if (qp->order < QW_ORDER_AUTO || qp->order > QW_ORDER_GIVEN)
            return arg_error("qw_run_workload: unknown order");
        if (qp->rerank < QW_RERANK_FP32 || qp->rerank > QW_RERANK_BF16_TC)
            return arg_error("qw_run_workload: unknown rerank");
        if (qp->start < QW_START_PLAIN || qp->start > QW_START_LEARNED)
            return arg_error("qw_run_workload: unknown start");
        if (qp->graph != 0 && qp->graph != 1) return arg_error("qw_run_workload: graph must be 0 or 1");
        if (qp->bitmap_loads != QW_LOADS_TMA && qp->bitmap_loads != QW_LOADS_DIRECT &&
            qp->bitmap_loads != QW_LOADS_FUSED)
            return arg_error("qw_run_workload: unknown bitmap_loads");
        if (qp->l2_mode < QW_L2_OFF || qp->l2_mode > QW_L2_MODEL)
            return arg_error("qw_run_workload: unknown l2_mode");
        if (qp->l2_index_permille < 0 || qp->l2_index_permille > 1000)
            return arg_error("qw_run_workload: l2_index_permille must be in [0, 1000]");
        if (qp->projection != QW_PROJ_FP32 && qp->projection != QW_PROJ_TENSOR)
            return arg_error("qw_run_workload: unknown projection");
        if (qp->probes < 0 || qp->probes > 64)
            return arg_error("qw_run_workload: probes must be in [0, 64]");
        if (qp->probes > 0 && (qp->path == QW_PATH_BITMAP || qp->path == QW_PATH_CLUSTER))
            return arg_error("qw_run_workload: multi-probe (probes > 0) runs on the level path");
        if (qp->rerank_rows != 0 && qp->rerank_rows != 2 && qp->rerank_rows != 4 &&
            qp->rerank_rows != 8)
            return arg_error("qw_run_workload: rerank_rows must be 0, 2, 4 or 8");
        if (qp->tiles_per_warp != 0 && qp->tiles_per_warp != 4 && qp->tiles_per_warp != 8 &&
            qp->tiles_per_warp != 16)
            return arg_error("qw_run_workload: tiles_per_warp must be 0, 4, 8 or 16");
        if (qp->projection == QW_PROJ_TENSOR && ix->m > 128)
            return arg_error("qw_run_workload: QW_PROJ_TENSOR needs m <= 128");
        if (ix->family == QW_FAMILY_QALSH) {
            if (qp->path == QW_PATH_BITMAP || qp->path == QW_PATH_CLUSTER)
                return arg_error("qw_run_workload: a QALSH index runs on the level path");
            if (qp->start == QW_START_LEARNED)
                return arg_error("qw_run_workload: learned start levels need the bucketed family");
            if (qp->probes > 0)
                return arg_error("qw_run_workload: multi-probe needs the bucketed family");
            if (qp->projection != QW_PROJ_FP32)
                return arg_error("qw_run_workload: a QALSH index projects queries in FP64 "
                                 "(projection must be QW_PROJ_FP32)");
        }
    }
    return QW_OK;
}

qw_status qw_run_workload(qw_index *ix, const float *queries, int64_t nq, int32_t k,
                          const qw_query_params *qp, int64_t *ids, float *dists, int64_t *stats,
                          int32_t mem, void *stream)
{
    clear_error();
    QW_TRY(check_workload_args(ix, queries, nq, k, qp, mem));
    if (nq > 0 && (!ids || !dists)) return arg_error("qw_run_workload: null output pointer");
    if (nq == 0) return QW_OK;
    return run_impl(ix, queries, nq, k, qp, ids, dists, stats, nullptr, nullptr, mem,
                    (cudaStream_t)stream);
}

qw_status qw_autotune(qw_index *ix, const float *queries, int64_t nq, int32_t k, int32_t mem,
                      int32_t reps, const qw_query_params *base, qw_query_params *best,
                      qw_tune_report *report, void *stream)
{
    clear_error();
    qw_query_params p0{};
    if (base) p0 = *base;
    p0.batch = 0;
    p0.path = QW_PATH_LEVELS;
    p0.order = QW_ORDER_SIGNATURE;
    p0.rerank = QW_RERANK_FP32;
    p0.start = QW_START_PLAIN;
    p0.graph = 0;
    p0.clusters = 0;
    p0.l2_mode = QW_L2_OFF;
    p0.l2_index_permille = 0;
    QW_TRY(check_workload_args(ix, queries, nq, k, &p0, mem));
    if (!best) return arg_error("qw_autotune: best is null");
    if (reps < 1) return arg_error("qw_autotune: reps < 1");
    if (nq < 1) return arg_error("qw_autotune: no queries");
    if (report) memset(report, 0, sizeof(*report));
    cudaStream_t s = (cudaStream_t)stream;
    const bool host = mem == QW_MEM_HOST;
    // results of every trial go to one device buffer (host mode: host buffer)
    DevBuf out_dev;
    std::vector<char> out_host;
    const size_t ob = (size_t)nq * k * (sizeof(int64_t) + sizeof(float));
    int64_t *ids;
    float *dists;
    if (host) {
        try {
            out_host.resize(ob);
        } catch (const std::bad_alloc &) {
            set_error("qw_autotune: out of host memory");
            return QW_ERR_OOM;
        }
        ids = reinterpret_cast<int64_t *>(out_host.data());
    } else {
        QW_TRY(out_dev.ensure(ob));
        ids = out_dev.as<int64_t>();
    }
    dists = reinterpret_cast<float *>(ids + (size_t)nq * k);
    cudaEvent_t e0, e1;
    QW_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_status(cudaErrorUnknown, "cudaEventCreate");
    }
    // the library's own batch choice for the level path, as the base of the batch sweep
    const int64_t wpq_bytes = (int64_t)ix->nT * kTile;
    const int64_t b_default =
        std::min<int64_t>(std::min<int64_t>(std::max<int64_t>(1, ((int64_t)2 << 30) / wpq_bytes), nq),
                          65535);
    const bool saved_tuned = ix->tuned;
    ix->tuned = false;  // trials name their path and batch explicitly
    int tried = 0;
    qw_status status = QW_OK;
    auto time_one = [&](const qw_query_params &p, float *ms_out) -> qw_status {
        QW_TRY(run_impl(ix, queries, nq, k, &p, ids, dists, nullptr, nullptr, nullptr, mem, s));
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            QW_CUDA_TRY(cudaEventRecord(e0, s));
            QW_TRY(run_impl(ix, queries, nq, k, &p, ids, dists, nullptr, nullptr, nullptr, mem, s));
            QW_CUDA_TRY(cudaEventRecord(e1, s));
            QW_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.0f;
            QW_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        *ms_out = t[t.size() / 2];
        if (report && tried < QW_TUNE_MAX) {
            report->params[tried] = p;
            report->ms[tried] = *ms_out;
        }
        ++tried;
        return QW_OK;
    };
    qw_query_params cur = p0;
    float cur_ms = 0.0f;
    int cur_slot = 0;
    // an alternative replaces the current setting only when it is more than
    // 1 % faster (trials differing by less than that are noise)
    auto try_alt = [&](const qw_query_params &alt) -> qw_status {
        float ms = 0.0f;
        const int slot = tried;
        QW_TRY(time_one(alt, &ms));
        if (ms < cur_ms * 0.99f) {
            cur = alt;
            cur_ms = ms;
            cur_slot = slot;
        }
        return QW_OK;
    };
    do {
        if ((status = time_one(cur, &cur_ms)) != QW_OK) break;
        int csize = 0, tpc = 0;
        // 1. first level
        if (ix->family == QW_FAMILY_E2LSH && ix->start_model &&
            mlp_inputs(ix->start_model) == ix->d + ix->m) {
            qw_query_params alt = cur;
            alt.start = QW_START_LEARNED;
            if ((status = try_alt(alt)) != QW_OK) break;
        }
        // 2. queries per batch and 3. graph mode, on the level path
        {
            const int64_t cands[3] = {b_default / 16, b_default / 4, b_default * 4};
            const qw_query_params keep = cur;
            for (int64_t bb : cands) {
                bb = std::min<int64_t>(std::min<int64_t>(bb, nq), 65535);
                if (bb < 1 || bb == b_default) continue;
                qw_query_params alt = keep;
                alt.batch = (int32_t)bb;
                if ((status = try_alt(alt)) != QW_OK) break;
            }
            if (status != QW_OK) break;
            qw_query_params alt = cur;
            alt.graph = 1;
            if ((status = try_alt(alt)) != QW_OK) break;
        }
        // 4. the bitmap path (when built): default batch, then its batch and graph
        //    (multi-probe runs on the level path only)
        if (ix->bitmaps && p0.probes == 0) {
            const qw_query_params best_levels = cur;
            const float best_levels_ms = cur_ms;
            const int best_levels_slot = cur_slot;
            qw_query_params bp0 = cur;
            bp0.path = QW_PATH_BITMAP;
            bp0.batch = 0;
            bp0.graph = 0;
            bp0.bitmap_loads = QW_LOADS_DIRECT;
            float bms = 0.0f;
            const int bslot = tried;
            if ((status = time_one(bp0, &bms)) != QW_OK) break;
            cur = bp0;
            cur_ms = bms;
            cur_slot = bslot;
            // the counting kernels first, then the batch size and graph mode
            // for the kernels chosen
            {
                const qw_query_params keepl = cur;
                for (int32_t ld : {QW_LOADS_TMA, QW_LOADS_FUSED}) {
                    qw_query_params alt = keepl;
                    alt.bitmap_loads = ld;
                    if ((status = try_alt(alt)) != QW_OK) break;
                }
                if (status != QW_OK) break;
            }
            const int64_t cb_b = (int64_t)ix->nT * kBmUint4 * (int64_t)sizeof(uint4) * 2 +
                                 (int64_t)ix->nT * (int64_t)sizeof(int32_t) * 2 +
                                 ((int64_t)kQCap * (int64_t)sizeof(uint64_t) + 4) * 2;
            const int64_t bdef = std::min<int64_t>(
                std::min<int64_t>(std::max<int64_t>(1, kBitmapBudget / cb_b), nq), 65535);
            const int64_t bc[2] = {bdef / 16, bdef / 4};
            const qw_query_params keepb = cur;
            for (int64_t bb : bc) {
                bb = std::min<int64_t>(std::min<int64_t>(bb, nq), 65535);
                if (bb < 1 || bb == bdef) continue;
                qw_query_params alt = keepb;
                alt.batch = (int32_t)bb;
                if ((status = try_alt(alt)) != QW_OK) break;
            }
            if (status != QW_OK) break;
            qw_query_params alt = cur;
            alt.graph = 1;
            if ((status = try_alt(alt)) != QW_OK) break;
            // tile shape of the filter / fused kernels: tiles per warp
            if (cur.bitmap_loads != QW_LOADS_TMA) {
                const qw_query_params keept = cur;
                for (int tw : {4, 16}) {
                    qw_query_params a2 = keept;
                    a2.tiles_per_warp = tw;
                    if ((status = try_alt(a2)) != QW_OK) break;
                }
                if (status != QW_OK) break;
            }
            if (best_levels_ms < cur_ms) {
                cur = best_levels;
                cur_ms = best_levels_ms;
                cur_slot = best_levels_slot;
            }
        }
        // 5. path: the cluster path (plain starts only) against the best so far
        if (ix->family == QW_FAMILY_E2LSH && cur.start == QW_START_PLAIN && cur.probes == 0 &&
            cluster_path_fits(ix->view(), &csize, &tpc)) {
            qw_query_params alt = cur;
            alt.path = QW_PATH_CLUSTER;
            alt.batch = 0;
            alt.graph = 0;
            if ((status = try_alt(alt)) != QW_OK) break;
        }
        // 6. order, 7. distance arithmetic
        {
            qw_query_params alt = cur;
            alt.order = QW_ORDER_GIVEN;
            if ((status = try_alt(alt)) != QW_OK) break;
        }
        if (ix->shadow) {
            const qw_query_params keepb = cur;
            for (int32_t mode : {QW_RERANK_BF16, QW_RERANK_BF16_TC}) {
                qw_query_params alt = keepb;
                alt.rerank = mode;
                if ((status = try_alt(alt)) != QW_OK) break;
            }
            if (status != QW_OK) break;
        }
        // tile shape of the rerank: candidate rows per warp
        {
            const qw_query_params keepr = cur;
            for (int rows : {2, 8}) {
                qw_query_params alt = keepr;
                alt.rerank_rows = rows;
                if ((status = try_alt(alt)) != QW_OK) break;
            }
            if (status != QW_OK) break;
        }
        // 8. the queries' projection on the tensor cores
        if (ix->family == QW_FAMILY_E2LSH && ix->m <= 128) {
            qw_query_params alt = cur;
            alt.projection = QW_PROJ_TENSOR;
            if ((status = try_alt(alt)) != QW_OK) break;
        }
        // 9. persisting-L2 windows split by the cost model
        {
            qw_query_params alt = cur;
            alt.l2_mode = QW_L2_MODEL;
            alt.l2_index_permille = 0;
            if ((status = try_alt(alt)) != QW_OK) break;
        }
    } while (false);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != QW_OK) {
        ix->tuned = saved_tuned;
        return status;
    }
    *best = cur;
    ix->tuned = true;
    ix->tuned_path = cur.path;
    ix->tuned_batch = cur.batch;
    if (report) {
        report->tried = std::min(tried, QW_TUNE_MAX);
        report->best = cur_slot < QW_TUNE_MAX ? cur_slot : -1;
    }
    return QW_OK;
}

qw_status qw_workload_candidates(qw_index *ix, const float *queries, int64_t nq, int32_t k,
                                 const qw_query_params *qp, int64_t *cand_ids, int32_t *cand_col,
                                 int64_t *stats, int32_t mem, void *stream)
{
    clear_error();
    QW_TRY(check_workload_args(ix, queries, nq, k, qp, mem));
    if (nq > 0 && !cand_ids) return arg_error("qw_workload_candidates: cand_ids is null");
    if (nq == 0) return QW_OK;
    return run_impl(ix, queries, nq, k, qp, nullptr, nullptr, stats, cand_ids, cand_col, mem,
                    (cudaStream_t)stream);
}

qw_status qw_query_features(qw_index *ix, const float *queries, int64_t nq, float *F, void *stream)
{
    clear_error();
    if (!ix || (nq > 0 && (!queries || !F))) return arg_error("qw_query_features: null pointer");
    if (nq < 0) return arg_error("qw_query_features: nq < 0");
    if (nq == 0) return QW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    QW_TRY(ix->w_hq.ensure((size_t)nq * ix->m * sizeof(int32_t)));
    QW_TRY(ix->w_err.ensure(128));
    int *err = ix->w_err.as<int>();
    QW_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    QW_TRY(launch_hash(queries, nq, ix->d, ix->A.as<float>(), ix->b.as<float>(), ix->m, ix->w,
                       ix->w_hq.as<int32_t>(), ix->m, 1, err, nullptr, s));
    QW_TRY(launch_features(queries, ix->w_hq.as<int32_t>(), nq, ix->view(), ix->xs, F, s));
    int h_err = 0;
    QW_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err & 2) {
        set_error("qw_query_features: a query bucket id falls outside int32");
        return QW_ERR_RANGE;
    }
    return QW_OK;
}

qw_status qw_index_set_start_model(qw_index *ix, qw_mlp *mlp, float eps)
{
    clear_error();
    if (!ix) return arg_error("qw_index_set_start_model: index is null");
    if (mlp) {
        if (!(eps > 0.0f && eps < 1.0f)) return arg_error("qw_index_set_start_model: eps not in (0, 1)");
        if (mlp_inputs(mlp) != ix->d + ix->m)
            return arg_error("qw_index_set_start_model: the model's input size is not d + m");
    }
    ix->start_model = mlp;
    ix->start_eps = eps;
    return QW_OK;
}

qw_status qw_index_profile(qw_index *ix, qw_profile *out, int32_t reset)
{
    clear_error();
    if (!ix || !out) return arg_error("qw_index_profile: null pointer");
    *out = ix->prof;
    if (reset) ix->prof = qw_profile{};
    return QW_OK;
}

qw_status qw_index_get_info(const qw_index *ix, qw_index_info *info)
{
    clear_error();
    if (!ix || !info) return arg_error("qw_index_get_info: null pointer");
    info->n = ix->n;
    info->d = ix->d;
    info->m = ix->m;
    info->w = ix->w;
    info->c = ix->c;
    info->v = ix->v;
    info->l = ix->l;
    info->tile = kTile;
    info->n_tiles = ix->nT;
    info->span_max = ix->span_max;
    info->n_fixups = ix->n_fixups;
    info->device_bytes = ix->device_bytes;
    info->bitmap_bytes = (int64_t)(ix->host_bitmaps ? ix->bm_host.bytes : ix->bm.bytes);
    info->host_bytes = (int64_t)ix->bm_host.bytes;
    info->family = ix->family;
    return QW_OK;
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) used as a counter-based generator: the value of
// counter k under `seed` is the mixing function applied to
// seed + (k + 1) * 0x9E3779B97F4A7C15.
static uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform double in [0, 1) from the top 53 bits.
static double uniform_at(uint64_t seed, uint64_t k)
{
    return (double)(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

void qw_draw_projections(uint64_t seed, int32_t m, int32_t d, float w, float *A, float *b)
{
    if (m < 1 || d < 1 || !A || !b) return;
    const uint64_t na = (uint64_t)m * (uint64_t)d;
    const double two_pi = 6.283185307179586476925286766559;
    // entries of A in row-major order, two per Box-Muller pair: entry e uses
    // the uniforms of counters 2 (e / 2) and 2 (e / 2) + 1
    for (uint64_t e = 0; e < na; e += 2) {
        const double u1 = uniform_at(seed, e);
        const double u2 = uniform_at(seed, e + 1);
        const double r = sqrt(-2.0 * log(1.0 - u1));
        const double t = two_pi * u2;
        A[e] = (float)(r * cos(t));
        if (e + 1 < na) A[e + 1] = (float)(r * sin(t));
    }
    // offsets from the counters after A's: b_i = u w, kept below w in float
    const uint64_t k0 = (na + 1) / 2 * 2;
    for (int32_t i = 0; i < m; ++i) {
        float bi = (float)(uniform_at(seed, k0 + (uint64_t)i) * (double)w);
        if (!(bi < w)) bi = nextafterf(w, 0.0f);
        b[i] = bi;
    }
}

qw_status qw_index_get_projections(const qw_index *ix, float *A, float *b, int32_t *offsets)
{
    clear_error();
    if (!ix) return arg_error("qw_index_get_projections: index is null");
    const int m = ix->m, d = ix->d;
    if (A) QW_CUDA_TRY(cudaMemcpy(A, ix->A.p, (size_t)m * d * sizeof(float), cudaMemcpyDeviceToHost));
    if (b) QW_CUDA_TRY(cudaMemcpy(b, ix->b.p, (size_t)m * sizeof(float), cudaMemcpyDeviceToHost));
    if (offsets)
        QW_CUDA_TRY(cudaMemcpy(offsets, ix->o.p, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return QW_OK;
}

qw_status qw_index_export(const qw_index *ix, int32_t *o, int32_t *span, int32_t *entry_bid,
                          int32_t *entry_id, void *stream)
{
    clear_error();
    if (!ix) return arg_error("qw_index_export: index is null");
    cudaStream_t s = (cudaStream_t)stream;
    const int m = ix->m;
    const int64_t n = ix->n;
    if (o) QW_CUDA_TRY(cudaMemcpyAsync(o, ix->o.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (span)
        QW_CUDA_TRY(cudaMemcpyAsync(span, ix->span.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if ((entry_bid || entry_id) && ix->family == QW_FAMILY_QALSH)
        return arg_error("qw_index_export: a QALSH index has no bucket ids");
    if (entry_bid || entry_id) {
        DevBuf eb, ei;
        if (entry_bid) QW_TRY(eb.ensure((size_t)m * n * sizeof(int32_t)));
        if (entry_id) QW_TRY(ei.ensure((size_t)m * n * sizeof(int32_t)));
        QW_TRY(launch_export(ix->lid.as<uint16_t>(), ix->dir_bid.as<int32_t>(),
                             ix->dir_off.as<int32_t>(), ix->dir_start.as<int64_t>(),
                             ix->dir_cnt.as<int32_t>(), n, m, ix->nT, eb.as<int32_t>(),
                             ei.as<int32_t>(), s));
        if (entry_bid)
            QW_CUDA_TRY(cudaMemcpyAsync(entry_bid, eb.p, (size_t)m * n * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, s));
        if (entry_id)
            QW_CUDA_TRY(cudaMemcpyAsync(entry_id, ei.p, (size_t)m * n * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, s));
        QW_CUDA_TRY(cudaStreamSynchronize(s));
        eb.release();
        ei.release();
    }
    QW_CUDA_TRY(cudaStreamSynchronize(s));
    return QW_OK;
}

void qw_index_free(qw_index *ix)
{
    if (!ix) return;
    cudaDeviceSynchronize();
    l2_release(&ix->l2_owner);
    ix->bm_host.release();
    DevBuf *bufs[] = {&ix->X, &ix->Xb, &ix->xnorm, &ix->Cg, &ix->Xcr, &ix->A, &ix->b, &ix->o, &ix->span, &ix->lid,
                      &ix->dir_bid,
                      &ix->dir_off, &ix->dir_start, &ix->dir_cnt, &ix->w_q, &ix->w_hq,
                      &ix->w_state, &ix->w_counters, &ix->w_cand, &ix->w_out, &ix->w_err,
                      &ix->w_order, &ix->w_qb, &ix->w_ob};
    for (DevBuf *bb : bufs) bb->release();
    DevBuf *bmb[] = {&ix->bm,  &ix->bm_base,    &ix->bm_nb,      &ix->bm_lvl,
                     &ix->bm_J, &ix->bid_prefix, &ix->prefix_off, &ix->w_cbits,
                     &ix->w_clist, &ix->perm, &ix->bm_sum, &ix->w_bmsel, &ix->w_ovf,
                     &ix->w_bmwork, &ix->w_rdstore, &ix->Xloc, &ix->inv, &ix->hloc,
                     &ix->qkey, &ix->qmin, &ix->qmax};
    for (DevBuf *bb : bmb) bb->release();
    for (cudaEvent_t e : ix->event_pool) cudaEventDestroy(e);
    level_graph_cache_free(ix->graphs);
    delete ix;
}

}  // extern "C"
