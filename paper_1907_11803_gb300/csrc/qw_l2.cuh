// qw_l2.cuh -- persisting-L2 windows of a workload call (see qw_l2.cu).
#pragma once

#include <algorithm>

#include "qw_internal.cuh"

namespace qw {

// One address range a window may cover, and the bytes the workload is
// expected to read from it.
struct L2Region {
    const void *base = nullptr;
    size_t bytes = 0;
    double reads = 0.0;
};

enum class L2Use { None, Index, Data };

// The context's persisting-L2 set-aside as an index found it: raised by the
// index's first call with windows, put back (and its persisting lines
// demoted) by l2_release when the index is freed.
struct L2Owner {
    bool raised = false;
    size_t old_limit = 0;
};
void l2_release(L2Owner *o);

// The windows of one qw_run_workload call.  begin() raises the set-aside
// (once per index) and saves the stream's window; end() (also run by the
// destructor, so every return path restores it) puts the stream's window back.
struct L2Session {
    bool on = false;
    size_t setaside = 0;
    int index_permille = 0;
    cudaAccessPolicyWindow win_index{}, win_data{};

    qw_status begin(L2Owner *owner, int mode, int permille, const L2Region &index,
                    const L2Region &data, cudaStream_t s);
    // Attach the index window, the data window or none to later launches on s.
    qw_status use(L2Use which, cudaStream_t s);
    cudaAccessPolicyWindow window(L2Use which) const;
    void end();
    ~L2Session() { end(); }

  private:
    static void make_window(const L2Region &r, double share, size_t max_window,
                            cudaAccessPolicyWindow *w);
    cudaStream_t stream = nullptr;
    cudaAccessPolicyWindow old_window{};
};

// Graph mode of the level loop (qw_graph.cu) with the access-policy window
// `win` on every kernel node of the batch's graph (num_bytes 0: none).
qw_status run_level_graph(LevelGraphCache *c, const IndexView &ix, int nb, int l, int cgrow,
                          int cap, bool learned, bool bitmap, int loads, int tpw, QueryState &st,
                          LoopCtl *ctl, int *err, cudaStream_t s,
                          const cudaAccessPolicyWindow &win);

// Eq. 4 restated for a hardware cache: the permille of the set-aside for the
// index region (see qw_l2_split_model in qwlsh.h); -1 on invalid arguments.
int32_t l2_split_model(double setaside, double index_bytes, double index_reads,
                       double data_bytes, double data_reads);

}  // namespace qw
