// Many realisations in one CUDA graph (poly_estimate_batched).
//
// The first call with a given (plans, fields, outputs) list captures every
// realisation's launches into one graph; later calls with the same list replay
// it with a single cudaGraphLaunch.  Realisations that share a plan share its
// workspace, so they stay in order on one branch of the graph; realisations of
// different plans (e.g. different grid sizes) run on parallel branches, forked
// from and joined back to the caller's stream, so their kernels can overlap on
// the GPU.  The results are those of the single-field calls, bit for bit: each
// realisation runs the same kernels with the same launch shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "plan_internal.h"

namespace {

struct BatchGraph {
    int device = -1;
    std::vector<const void*> key;  // plans, fields, outputs
    cudaGraphExec_t exec = nullptr;
    unsigned long long last_use = 0;
};

constexpr size_t kMaxGraphs = 8;
std::mutex g_mu;
std::vector<BatchGraph> g_graphs;
unsigned long long g_clock = 0;

poly_status fail(poly_status s, const std::string& msg) {
    ps_set_last_error(msg);
    return s;
}

void destroy(BatchGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
}

// Capture the realisations into an executable graph.  On failure nothing is left
// capturing and no graph is returned.
poly_status capture(const poly_plan* plans, const void* const* fields, double* const* outs, int count,
                    cudaGraphExec_t* exec_out) {
    *exec_out = nullptr;
    // one branch per distinct plan, in order of first appearance
    std::vector<PsPlan*> distinct;
    std::vector<int> branch(count);
    for (int i = 0; i < count; i++) {
        auto it = std::find(distinct.begin(), distinct.end(), plans[i]);
        branch[i] = (int)(it - distinct.begin());
        if (it == distinct.end()) distinct.push_back(plans[i]);
    }
    const int nb = (int)distinct.size();
    std::vector<cudaStream_t> streams(nb + 1, nullptr);
    std::vector<cudaEvent_t> events(nb + 1, nullptr);
    poly_status s = POLY_OK;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b <= nb && !e; b++) {
        e = cudaStreamCreateWithFlags(&streams[b], cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&events[b], cudaEventDisableTiming);
    }
    if (e) s = fail(POLY_ERR_CUDA, std::string("stream or event for graph capture: ") + cudaGetErrorString(e));
    cudaGraph_t graph = nullptr;
    bool capturing = false;
    if (!s) {
        // streams[0] is the origin; branch b runs on streams[b + 1]
        e = cudaStreamBeginCapture(streams[0], cudaStreamCaptureModeThreadLocal);
        if (e) s = fail(POLY_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
        else capturing = true;
    }
    if (!s && (e = cudaEventRecord(events[0], streams[0])))
        s = fail(POLY_ERR_CUDA, std::string("fork event: ") + cudaGetErrorString(e));
    for (int b = 0; b < nb && !s; b++)
        if ((e = cudaStreamWaitEvent(streams[b + 1], events[0], 0)))
            s = fail(POLY_ERR_CUDA, std::string("fork: ") + cudaGetErrorString(e));
    for (int i = 0; i < count && !s; i++) {
        PsPlan* p = plans[i];
        const bool timing = p->timing;
        p->timing = false;  // no event records inside the graph
        s = ps_estimate_impl(p, fields[i], outs[i], nullptr, streams[branch[i] + 1]);
        p->timing = timing;
    }
    for (int b = 0; b < nb && !s; b++) {
        if ((e = cudaEventRecord(events[b + 1], streams[b + 1])) || (e = cudaStreamWaitEvent(streams[0], events[b + 1], 0)))
            s = fail(POLY_ERR_CUDA, std::string("join: ") + cudaGetErrorString(e));
    }
    if (capturing) {
        e = cudaStreamEndCapture(streams[0], &graph);
        if (!s && e) s = fail(POLY_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    if (!s && (e = cudaGraphInstantiate(exec_out, graph, 0)))
        s = fail(POLY_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    if (graph) cudaGraphDestroy(graph);
    for (int b = 0; b <= nb; b++) {
        if (events[b]) cudaEventDestroy(events[b]);
        if (streams[b]) cudaStreamDestroy(streams[b]);
    }
    if (s) {
        if (*exec_out) cudaGraphExecDestroy(*exec_out);
        *exec_out = nullptr;
        cudaGetLastError();
    }
    return s;
}

}  // namespace

poly_status ps_batched_impl(const poly_plan* plans, const void* const* fields, double* const* outs, int count,
                            cudaStream_t st) {
    if (count < 0 || (count > 0 && (!plans || !fields || !outs))) return fail(POLY_ERR_ARG, "NULL argument");
    if (count == 0) return POLY_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    for (int i = 0; i < count; i++) {
        if (!plans[i] || !fields[i] || !outs[i]) return fail(POLY_ERR_ARG, "NULL plan, field or output");
        if (plans[i]->device != dev) return fail(POLY_ERR_ARG, "every plan must live on the current device");
    }
    std::vector<const void*> key;
    key.reserve(3 * (size_t)count);
    for (int i = 0; i < count; i++) key.push_back(plans[i]);
    for (int i = 0; i < count; i++) key.push_back(fields[i]);
    for (int i = 0; i < count; i++) key.push_back(outs[i]);
    std::lock_guard<std::mutex> lk(g_mu);
    BatchGraph* g = nullptr;
    for (auto& c : g_graphs)
        if (c.device == dev && c.key == key) g = &c;
    if (!g) {
        cudaGraphExec_t exec = nullptr;
        poly_status s = capture(plans, fields, outs, count, &exec);
        if (s) return s;
        if (g_graphs.size() >= kMaxGraphs) {
            auto lru = std::min_element(g_graphs.begin(), g_graphs.end(),
                                        [](const BatchGraph& a, const BatchGraph& b) { return a.last_use < b.last_use; });
            destroy(*lru);
            g_graphs.erase(lru);
        }
        g_graphs.push_back(BatchGraph{dev, std::move(key), exec, 0});
        g = &g_graphs.back();
    }
    g->last_use = ++g_clock;
    cudaError_t e = cudaGraphLaunch(g->exec, st);
    if (e) return fail(POLY_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return POLY_OK;
}

// Drop every cached graph that references plan p (called before p is destroyed).
void ps_batched_forget(const PsPlan* p) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_graphs.size();) {
        if (std::find(g_graphs[i].key.begin(), g_graphs[i].key.end(), (const void*)p) != g_graphs[i].key.end()) {
            destroy(g_graphs[i]);
            g_graphs.erase(g_graphs.begin() + (long)i);
        } else {
            i++;
        }
    }
}
