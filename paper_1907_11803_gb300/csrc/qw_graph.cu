// qw_graph.cu -- graph mode of the level loop.
//
// On the level path the host normally drives the collision-counting loop: it
// reads the batch's largest useful radius, launches one counting kernel and
// one decision kernel per level, and (learned start) reads how many queries
// must be recomputed.  Each of those reads is a stream synchronisation.  In
// graph mode the whole loop of one batch is a CUDA graph whose level loop is
// a conditional WHILE node: the body counts one level, decides, and a
// one-thread kernel advances the level on the device and sets the loop
// condition.  With learned start a second WHILE node recomputes the queries
// that stopped at their learned first level.  One graph launch per batch, no
// host synchronisation inside the batch; the kernels and their order are
// those of the host loop, so the results are the same.
//
// Graphs are cached per batch shape (batch size, every workspace pointer the
// kernels take, and the index's parameters) and per persisting-L2 window: a
// workload of full batches and one short batch instantiates two graphs on its
// first call and none afterwards.  The window (see qw_l2.cu) is set on every
// kernel node of the graph, loop bodies included.
#include "qw_internal.cuh"
#include "qw_l2.cuh"

#include <string.h>

#include <vector>

namespace qw {

struct GraphKey {
    int nb, l, cgrow, cap;
    bool learned, bitmap;
    int loads, tpw;
    QueryState st;         // every workspace pointer the graph's kernels take by value
    const void *lid;       // the index
    const void *ctl;
    const void *err;
    const void *win_base;  // persisting-L2 window of the kernel nodes
    size_t win_bytes;
    float win_hit;
    bool operator==(const GraphKey &o) const
    {
        return nb == o.nb && l == o.l && cgrow == o.cgrow && cap == o.cap &&
               learned == o.learned && bitmap == o.bitmap && loads == o.loads && tpw == o.tpw &&
               memcmp(&st, &o.st, sizeof(QueryState)) == 0 && lid == o.lid && ctl == o.ctl &&
               err == o.err && win_base == o.win_base && win_bytes == o.win_bytes &&
               win_hit == o.win_hit;
    }
};

struct LevelGraphCache {
    cudaStream_t cap_stream = nullptr;  // private stream used only for capture
    struct Entry {
        GraphKey key;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
    };
    std::vector<Entry> entries;
};

LevelGraphCache *level_graph_cache_new() { return new (std::nothrow) LevelGraphCache(); }

void level_graph_cache_free(LevelGraphCache *c)
{
    if (!c) return;
    for (auto &e : c->entries) {
        cudaGraphExecDestroy(e.exec);
        cudaGraphDestroy(e.graph);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

namespace {

// Capture kernels launched by f into graph g after the nodes deps; returns
// the graph's sink node in *last (the capture must end in one node).
template <class F>
qw_status capture_into(cudaStream_t cs, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                       F &&f)
{
    QW_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, g, deps, nullptr, ndeps,
                                              cudaStreamCaptureModeThreadLocal));
    const qw_status st = f();
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &out);
    QW_TRY(st);
    QW_CUDA_TRY(e);
    return QW_OK;
}

// Nodes of g that no other node depends on.
qw_status sinks(cudaGraph_t g, std::vector<cudaGraphNode_t> &out)
{
    size_t n = 0;
    QW_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    QW_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &n));
    out.clear();
    for (cudaGraphNode_t nd : nodes) {
        size_t nout = 0;
        QW_CUDA_TRY(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout));
        if (nout == 0) out.push_back(nd);
    }
    return QW_OK;
}

// Set the access-policy window on every kernel node of g (num_bytes 0
// clears it).
qw_status set_window(cudaGraph_t g, const cudaAccessPolicyWindow &win)
{
    size_t n = 0;
    QW_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    QW_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &n));
    cudaKernelNodeAttrValue v{};
    v.accessPolicyWindow = win;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        QW_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
        if (t == cudaGraphNodeTypeKernel)
            QW_CUDA_TRY(cudaGraphKernelNodeSetAttribute(
                nd, cudaKernelNodeAttributeAccessPolicyWindow, &v));
    }
    return QW_OK;
}

qw_status add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps,
                    cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    QW_CUDA_TRY(cudaGraphAddNode(&node, g, deps.data(), nullptr, deps.size(), &p));
    *body = p.conditional.phGraph_out[0];
    return QW_OK;
}

qw_status build(LevelGraphCache *c, const GraphKey &key, const IndexView &ix, int nb, int l,
                int cgrow, int cap, bool learned, bool bitmap, int loads, int tpw, QueryState &st,
                LoopCtl *ctl, int *err, const cudaAccessPolicyWindow &win,
                cudaGraph_t *graph_out)
{
    cudaStream_t cs = c->cap_stream;
    cudaGraph_t g = nullptr;
    QW_CUDA_TRY(cudaGraphCreate(&g, 0));
    auto fail = [&](qw_status s) {
        cudaGraphDestroy(g);
        return s;
    };
    // loop 1: from level 0 (each query's own first level when learned)
    cudaGraphConditionalHandle h1, h2;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h1, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail(cuda_status(e, "cudaGraphConditionalHandleCreate"));
    qw_status s =
        capture_into(cs, g, nullptr, 0, [&] { return launch_loop_init(ctl, st, nb, cgrow, cs); });
    if (s != QW_OK) return fail(s);
    std::vector<cudaGraphNode_t> tail;
    if ((s = sinks(g, tail)) != QW_OK) return fail(s);
    cudaGraph_t body;
    if ((s = add_while(g, tail, h1, &body)) != QW_OK) return fail(s);
    auto level_body = [&](cudaGraphConditionalHandle h) {
        return [&, h] {
            if (bitmap)
                QW_TRY(launch_bm_level(ix, nb, 0, 1, 1, l, cgrow, st, err, loads, cs, ctl, 0, tpw));
            else
                QW_TRY(launch_level(ix, nb, 0, 1, 1, l, cgrow, st, cs, ctl));
            ScanStats ss = bitmap ? scan_stats_of(ix, cgrow) : ScanStats();
            ss.recount_first = bitmap && learned;
            QW_TRY(launch_decide(nb, 0, 1, cap, st, cs, ctl, ss));
            return launch_loop_ctl(ctl, st.max_top, cgrow, h, err, cs);
        };
    };
    if ((s = capture_into(cs, body, nullptr, 0, level_body(h1))) != QW_OK) return fail(s);
    if (win.num_bytes > 0 && (s = set_window(body, win)) != QW_OK) return fail(s);
    if (learned) {
        // loop 2: the queries that stopped at their learned first level, from level 0
        e = cudaGraphConditionalHandleCreate(&h2, g, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return fail(cuda_status(e, "cudaGraphConditionalHandleCreate"));
        if ((s = sinks(g, tail)) != QW_OK) return fail(s);
        s = capture_into(cs, g, tail.data(), tail.size(),
                         [&] { return launch_fallback_graph(nb, st, ctl, h2, cs); });
        if (s != QW_OK) return fail(s);
        if ((s = sinks(g, tail)) != QW_OK) return fail(s);
        cudaGraph_t body2;
        if ((s = add_while(g, tail, h2, &body2)) != QW_OK) return fail(s);
        if ((s = capture_into(cs, body2, nullptr, 0, level_body(h2))) != QW_OK) return fail(s);
        if (win.num_bytes > 0 && (s = set_window(body2, win)) != QW_OK) return fail(s);
    }
    if (win.num_bytes > 0 && (s = set_window(g, win)) != QW_OK) return fail(s);
    (void)key;
    *graph_out = g;
    return QW_OK;
}

}  // namespace

qw_status run_level_graph(LevelGraphCache *c, const IndexView &ix, int nb, int l, int cgrow,
                          int cap, bool learned, bool bitmap, int loads, int tpw, QueryState &st,
                          LoopCtl *ctl, int *err, cudaStream_t s)
{
    return run_level_graph(c, ix, nb, l, cgrow, cap, learned, bitmap, loads, tpw, st, ctl, err, s,
                           cudaAccessPolicyWindow{});
}

qw_status run_level_graph(LevelGraphCache *c, const IndexView &ix, int nb, int l, int cgrow,
                          int cap, bool learned, bool bitmap, int loads, int tpw, QueryState &st,
                          LoopCtl *ctl, int *err, cudaStream_t s,
                          const cudaAccessPolicyWindow &win)
{
    if (!c) {
        set_error("internal: no graph cache");
        return QW_ERR_CUDA;
    }
    GraphKey key;
    memset(&key, 0, sizeof(key));  // padding too: the key is compared bytewise in part
    key.nb = nb;
    key.l = l;
    key.cgrow = cgrow;
    key.cap = cap;
    key.learned = learned;
    key.bitmap = bitmap;
    key.loads = loads;
    key.tpw = tpw;
    key.st = st;
    key.lid = ix.lid;
    key.ctl = ctl;
    key.err = err;
    if (win.num_bytes > 0) {
        key.win_base = win.base_ptr;
        key.win_bytes = win.num_bytes;
        key.win_hit = win.hitRatio;
    }
    for (auto &en : c->entries)
        if (en.key == key) {
            QW_CUDA_TRY(cudaGraphLaunch(en.exec, s));
            return QW_OK;
        }
    if (!c->cap_stream) QW_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (c->entries.size() >= 8) {  // a few batch shapes at a time; drop the oldest
        cudaGraphExecDestroy(c->entries.front().exec);
        cudaGraphDestroy(c->entries.front().graph);
        c->entries.erase(c->entries.begin());
    }
    cudaGraph_t g = nullptr;
    QW_TRY(build(c, key, ix, nb, l, cgrow, cap, learned, bitmap, loads, tpw, st, ctl, err, win, &g));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_status(e, "cudaGraphInstantiate");
    }
    c->entries.push_back({key, g, ex});
    QW_CUDA_TRY(cudaGraphLaunch(ex, s));
    return QW_OK;
}

}  // namespace qw
