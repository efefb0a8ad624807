// batch.cpp -- many independent structures at once (unevenly sized voxel grids).
//
// A batch borrows handles that each hold one structure (grid, ports, kernel
// spectra). svh_batch_matvec applies every structure's operator to its own
// vectors: on the first call with a given argument set the launch sequences
// of all structures are captured into one CUDA graph, and that call and every
// later call with the same arguments replay it as a single graph launch (no
// per-kernel launch overhead for the hundreds of small kernels of a batch of
// small grids). The structures are spread over up to 16 lanes (streams forked
// from and joined to the batch stream), so the graph holds independent chains
// and the small products of different structures run concurrently. svh_batch_solve solves every
// structure's ports at the given frequencies with worker threads, each
// driving one structure at a time on its own stream, so that the host AMG of
// one structure overlaps the device work of the others.
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "svh_internal.h"

namespace svh {

struct Batch {
    int device = 0;
    cudaStream_t stream = nullptr;    // capture / replay stream (owned)
    static constexpr int kLanes = 16;
    std::vector<cudaStream_t> lanes;  // structure i runs on lanes[i % lanes.size()]
    std::vector<cudaEvent_t> lane_done;
    cudaEvent_t fork = nullptr;
    std::vector<Handle*> items;
    std::string err;
    // captured product
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key_x;
    std::vector<void*> key_y;
    std::vector<double> key_om;
    int key_nb = 0, key_prec = -1;
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        key_x.clear();
    }
};

static int berr(Batch* b, int code, const std::string& m) {
    b->err = m;
    return code;
}

static bool ensure_lanes(Batch* b) {
    const size_t want = std::min<size_t>(Batch::kLanes, std::max<size_t>(1, b->items.size()));
    if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return false;
    while (b->lanes.size() < want) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(st);
            return false;
        }
        b->lanes.push_back(st);
        b->lane_done.push_back(ev);
    }
    return true;
}

// every structure's product on its lane, forked from and joined to the batch stream
static int launch_all(Batch* b, const double* omegas, int nb, const void* const* x_dev, void* const* y_dev,
                      int precision, std::string& msg) {
    const size_t n = b->items.size(), L = std::min(b->lanes.size(), n);
    if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return SVH_ERR_CUDA;
    for (size_t l = 0; l < L; ++l)
        if (cudaStreamWaitEvent(b->lanes[l], b->fork, 0) != cudaSuccess) return SVH_ERR_CUDA;
    int rc = SVH_OK;
    for (size_t i = 0; i < n && rc == SVH_OK; ++i) {
        Handle* h = b->items[i];
        cudaStream_t saved = h->stream;
        h->stream = b->lanes[i % L];
        rc = precision == SVH_FP32 ? launch_matvec32(h, omegas[i], nb, x_dev[i], y_dev[i], 0)
                                   : launch_matvec64(h, omegas[i], nb, x_dev[i], y_dev[i], 0);
        if (rc) msg = h->err;
        h->stream = saved;
    }
    for (size_t l = 0; l < L; ++l) {
        cudaEventRecord(b->lane_done[l], b->lanes[l]);
        cudaStreamWaitEvent(b->stream, b->lane_done[l], 0);
    }
    return rc;
}

}  // namespace svh

using namespace svh;

extern "C" {

int svh_batch_create(svh_batch** out, int device) {
    if (!out) return SVH_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return SVH_ERR_CUDA;
    Batch* b = new (std::nothrow) Batch();
    if (!b) return SVH_ERR_OOM;
    b->device = device;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return SVH_ERR_CUDA;
    }
    *out = reinterpret_cast<svh_batch*>(b);
    return SVH_OK;
}

int svh_batch_destroy(svh_batch* bb) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return SVH_ERR_ARG;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->drop_graph();
    for (cudaStream_t st : b->lanes) cudaStreamDestroy(st);
    for (cudaEvent_t e : b->lane_done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaStreamDestroy(b->stream);
    delete b;
    return SVH_OK;
}

const char* svh_batch_last_error(const svh_batch* bb) {
    const Batch* b = reinterpret_cast<const Batch*>(bb);
    return b ? b->err.c_str() : "null batch";
}

int svh_batch_add(svh_batch* bb, svh_handle* hh) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!b || !h) return SVH_ERR_ARG;
    if (h->device != b->device) return berr(b, SVH_ERR_ARG, "svh_batch_add: handle on another device");
    if (!h->have_grid || !h->have_kernels) return berr(b, SVH_ERR_STATE, "svh_batch_add: handle needs grid and kernels");
    if (std::find(b->items.begin(), b->items.end(), h) != b->items.end())
        return berr(b, SVH_ERR_ARG, "svh_batch_add: handle already in the batch");
    b->items.push_back(h);
    b->drop_graph();
    return SVH_OK;
}

int svh_batch_size(const svh_batch* bb) {
    const Batch* b = reinterpret_cast<const Batch*>(bb);
    return b ? (int)b->items.size() : -1;
}

int svh_batch_matvec(svh_batch* bb, const double* omegas, int nb, const void* const* x_dev, void* const* y_dev,
                     int precision) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || !omegas || !x_dev || !y_dev || nb <= 0 || (precision != SVH_FP32 && precision != SVH_FP64))
        return b ? berr(b, SVH_ERR_ARG, "svh_batch_matvec: bad arguments") : SVH_ERR_ARG;
    if (b->items.empty()) return berr(b, SVH_ERR_STATE, "svh_batch_matvec: empty batch");
    if (cudaSetDevice(b->device) != cudaSuccess) return berr(b, SVH_ERR_CUDA, "cudaSetDevice failed");
    const size_t n = b->items.size();
    for (size_t i = 0; i < n; ++i)
        if (!(omegas[i] > 0) || !x_dev[i] || !y_dev[i]) return berr(b, SVH_ERR_ARG, "svh_batch_matvec: bad item arguments");
    const bool same = b->exec && b->key_nb == nb && b->key_prec == precision &&
                      std::equal(b->key_x.begin(), b->key_x.end(), x_dev) && b->key_x.size() == n &&
                      std::equal(b->key_y.begin(), b->key_y.end(), y_dev) &&
                      std::equal(b->key_om.begin(), b->key_om.end(), omegas);
    if (!same) {
        b->drop_graph();
        if (!ensure_lanes(b)) return berr(b, SVH_ERR_CUDA, "svh_batch_matvec: stream set-up failed");
        // run once eagerly so that every buffer a product needs exists before capture
        std::string msg;
        int rc = launch_all(b, omegas, nb, x_dev, y_dev, precision, msg);
        if (rc) return berr(b, rc, std::string("svh_batch_matvec: item product failed: ") + msg);
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return berr(b, SVH_ERR_CUDA, "svh_batch_matvec: eager run failed");
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            rc = launch_all(b, omegas, nb, x_dev, y_dev, precision, msg);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e2 == cudaSuccess && rc == SVH_OK) {
                b->graph = g;
                e2 = cudaGraphInstantiate(&b->exec, g, 0);
            } else if (g) {
                cudaGraphDestroy(g);
            }
            if (e2 != cudaSuccess) e = e2;
        }
        if (e != cudaSuccess || rc != SVH_OK) {
            b->drop_graph();
            cudaGetLastError();
            return berr(b, rc ? rc : SVH_ERR_CUDA, std::string("svh_batch_matvec: graph capture failed: ") +
                                                       (rc ? msg : std::string(cudaGetErrorString(e))));
        }
        b->key_x.assign(x_dev, x_dev + n);
        b->key_y.assign(y_dev, y_dev + n);
        b->key_om.assign(omegas, omegas + n);
        b->key_nb = nb;
        b->key_prec = precision;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return berr(b, SVH_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return SVH_OK;
}

int svh_batch_sync(svh_batch* bb) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return SVH_ERR_ARG;
    cudaSetDevice(b->device);
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? SVH_OK : SVH_ERR_CUDA;
}

void* svh_batch_stream(svh_batch* bb) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    return b ? static_cast<void*>(b->stream) : nullptr;
}

int svh_batch_solve(svh_batch* bb, const double* omegas, int nfreq, const svh_options* opt, double* const* Zports,
                    double* const* Lports, int n_workers, svh_stats* st) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || !omegas || nfreq <= 0 || !Zports) return b ? berr(b, SVH_ERR_ARG, "svh_batch_solve: bad arguments") : SVH_ERR_ARG;
    const int n = (int)b->items.size();
    if (n == 0) return berr(b, SVH_ERR_STATE, "svh_batch_solve: empty batch");
    const int workers = std::max(1, std::min(n_workers > 0 ? n_workers : 4, n));
    std::vector<int> rcs(n, SVH_OK);
    std::vector<svh_stats> sts(n);
    std::atomic<int> next(0);
    const int cores = std::max(1, omp_get_num_procs());
    const auto t0 = std::chrono::steady_clock::now();
    auto work = [&]() {
        cudaSetDevice(b->device);
        omp_set_num_threads(std::max(1, cores / workers));
        cudaStream_t s = nullptr;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        for (int i = next++; i < n; i = next++) {
            Handle* h = b->items[i];
            cudaStream_t saved = h->stream;
            h->stream = s;
            std::memset(&sts[i], 0, sizeof(svh_stats));
            rcs[i] = svh_solve(reinterpret_cast<svh_handle*>(h), omegas, nfreq, opt, Zports[i],
                               Lports ? Lports[i] : nullptr, &sts[i]);
            cudaStreamSynchronize(s);
            h->stream = saved;
        }
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w) pool.emplace_back(work);
    for (auto& t : pool) t.join();
    int status = SVH_OK;
    if (st) std::memset(st, 0, sizeof(svh_stats));
    for (int i = 0; i < n; ++i) {
        if (rcs[i] != SVH_OK && status == SVH_OK) {
            status = rcs[i];
            b->err = "svh_batch_solve: item " + std::to_string(i) + ": " + b->items[i]->err;
        }
        if (st) {
            st->iterations += sts[i].iterations;
            st->refinements += sts[i].refinements;
            st->amg_levels = std::max(st->amg_levels, sts[i].amg_levels);
            st->amg_avg_iterations += sts[i].amg_avg_iterations / n;
            st->final_rre = std::max(st->final_rre, sts[i].final_rre);
            st->setup_seconds += sts[i].setup_seconds;
        }
    }
    if (st) st->solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

}  // extern "C"
