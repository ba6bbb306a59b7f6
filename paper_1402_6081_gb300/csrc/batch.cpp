// Batched solves: many independent plans executed together.
//
// A batch forks the caller's stream into a pool of streams, issues each
// plan's solve (lgf_solve) on a pool stream round-robin, so small solves
// overlap on the device, and joins the pool back into the caller's stream.
// With use_graph the whole batch (every kernel of every solve, the forks and
// joins) is captured once into a CUDA graph and replayed by each launch, which
// removes the host launch cost of the few hundred small kernels of a batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lgf_internal.h"

struct lgf_batch_s {
    int device = 0;
    std::vector<lgf_plan> plans;
    std::vector<const void*> f;
    std::vector<void*> u;
    std::vector<cudaStream_t> pool;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaStream_t origin = nullptr;     // capture stream
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;

    ~lgf_batch_s() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaStream_t s : pool) cudaStreamDestroy(s);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (origin) cudaStreamDestroy(origin);
        cudaSetDevice(cur);
    }
};

namespace lgf {
namespace {

lgf_status cerr(cudaError_t e, const char* what) {
    return fail(LGF_ERR_CUDA, std::string("batch: ") + what + ": " + cudaGetErrorString(e));
}

// fork st into the pool, one solve per plan, join back into st
lgf_status issue(lgf_batch_s* B, cudaStream_t st) {
    cudaError_t e = cudaEventRecord(B->fork, st);
    if (e != cudaSuccess) return cerr(e, "fork");
    for (cudaStream_t s : B->pool)
        if ((e = cudaStreamWaitEvent(s, B->fork, 0)) != cudaSuccess) return cerr(e, "fork");
    for (size_t i = 0; i < B->plans.size(); ++i) {
        lgf_status r = lgf_solve(B->plans[i], B->f[i], B->u[i], B->pool[i % B->pool.size()]);
        if (r != LGF_OK) return r;
    }
    for (size_t k = 0; k < B->pool.size(); ++k) {
        if ((e = cudaEventRecord(B->join[k], B->pool[k])) != cudaSuccess) return cerr(e, "join");
        if ((e = cudaStreamWaitEvent(st, B->join[k], 0)) != cudaSuccess) return cerr(e, "join");
    }
    return ok();
}

}  // namespace
}  // namespace lgf

using namespace lgf;

extern "C" lgf_status lgf_batch_create(const lgf_plan* plans, const void* const* f_dev, void* const* u_dev, int32_t n,
                                       int32_t use_graph, lgf_batch* out) {
    if (!out || n < 1 || !plans || !f_dev || !u_dev)
        return fail(LGF_ERR_INVALID_ARG, "lgf_batch_create: need n >= 1 plans, inputs, outputs and out");
    *out = nullptr;
    for (int32_t i = 0; i < n; ++i) {
        if (!plans[i] || !f_dev[i] || !u_dev[i]) return fail(LGF_ERR_INVALID_ARG, "lgf_batch_create: NULL entry");
        for (int32_t j = 0; j < i; ++j)
            if (plans[i] == plans[j]) return fail(LGF_ERR_INVALID_ARG, "lgf_batch_create: plans must be distinct");
        // timing events recorded inside a capture belong to the graph and
        // cannot be read back per launch
        if (use_graph && plan_timing_capacity(plans[i]) > 0)
            return fail(LGF_ERR_INVALID_ARG, "lgf_batch_create: turn plan timing off before capturing a graph");
    }
    auto B = std::make_unique<lgf_batch_s>();
    cudaError_t e = cudaGetDevice(&B->device);
    if (e != cudaSuccess) return cerr(e, "cudaGetDevice");
    B->plans.assign(plans, plans + n);
    B->f.assign(f_dev, f_dev + n);
    B->u.assign(u_dev, u_dev + n);
    const int k = std::min<int>(n, 16);
    B->pool.resize(size_t(k));
    B->join.resize(size_t(k));
    for (int i = 0; i < k; ++i) {
        if ((e = cudaStreamCreateWithFlags(&B->pool[size_t(i)], cudaStreamNonBlocking)) != cudaSuccess)
            return cerr(e, "stream");
        if ((e = cudaEventCreateWithFlags(&B->join[size_t(i)], cudaEventDisableTiming)) != cudaSuccess)
            return cerr(e, "event");
    }
    if ((e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming)) != cudaSuccess) return cerr(e, "event");
    if (use_graph) {
        if ((e = cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking)) != cudaSuccess) return cerr(e, "stream");
        // one solve of each plan before capture: first-use work (function
        // attributes, lazy module loading) must not happen inside the capture
        lgf_status r = issue(B.get(), B->origin);
        if (r != LGF_OK) return r;
        if ((e = cudaStreamSynchronize(B->origin)) != cudaSuccess) return cerr(e, "warm-up");
        if ((e = cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cerr(e, "begin capture");
        r = issue(B.get(), B->origin);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(B->origin, &g);
        if (r != LGF_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e2 != cudaSuccess) return cerr(e2, "end capture");
        B->graph = g;
        if ((e = cudaGraphInstantiate(&B->exec, g, 0)) != cudaSuccess) return cerr(e, "instantiate");
    }
    *out = B.release();
    return ok();
}

extern "C" lgf_status lgf_batch_launch(lgf_batch batch, void* stream) {
    if (!batch) return fail(LGF_ERR_INVALID_ARG, "lgf_batch_launch: NULL batch");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != batch->device) return fail(LGF_ERR_INVALID_ARG, "lgf_batch_launch: batch belongs to another device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (batch->exec) {
        cudaError_t e = cudaGraphLaunch(batch->exec, st);
        return e == cudaSuccess ? ok() : cerr(e, "graph launch");
    }
    return issue(batch, st);
}

extern "C" lgf_status lgf_batch_destroy(lgf_batch batch) {
    if (!batch) return fail(LGF_ERR_INVALID_ARG, "lgf_batch_destroy: NULL batch");
    cudaSetDevice(batch->device);
    cudaDeviceSynchronize();
    delete batch;
    return ok();
}
