// batch.cpp -- many independent structures at once (unevenly sized voxel grids).
//
// A batch borrows handles that each hold one structure (grid, ports, kernel
// spectra). svh_batch_matvec applies every structure's operator to its own
// right-hand sides (any number per structure, each with its own frequency) in
// ONE persistent launch (batch_persist.cu): a device work queue of the tiles of
// every pass of every structure, taken by a grid sized to fill the GPU, with
// bounded waits for the passes each tile depends on. On the first call with a
// given argument set the queue is built and the launch (a counter reset and
// the kernel) is captured into a CUDA graph; that call and every later call
// with the same arguments replay the graph. svh_batch_solve solves every
// structure's ports at the given frequencies with worker threads, each
// driving one structure at a time on its own stream, so that the host AMG of
// one structure overlaps the device work of the others.
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "batch_persist.h"
#include "svh_internal.h"

namespace svh {

struct Batch {
    int device = 0;
    cudaStream_t stream = nullptr;    // capture / replay stream (owned)
    std::vector<Handle*> items;
    std::string err;
    // the queue of the current argument set (device arrays owned by the batch)
    DevBuf d_items, d_seg, d_segpi, d_cnt, d_status, d_omegas;
    BQueue q{};
    size_t smem = 0;
    int grid = 0;
    double wait_ms = 1000.0;          // bound of each dependency wait
    int hold_item = -1, hold_phase = -1;
    // mode 1: every structure's own launch sequence (size-specialised kernels, tuned tiles) on
    // up to kLanes streams forked from and joined to the batch stream, captured as one graph
    int mode = 0;
    static constexpr int kLanes = 16;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_done;
    cudaEvent_t fork = nullptr;
    // captured launch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key_x;
    std::vector<void*> key_y;
    std::vector<int32_t> key_nb;
    std::vector<double> key_om;
    int key_prec = -1, key_mode = -1;
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

// a Handle-free device upload for the batch's own arrays
static int bupload(Batch* b, DevBuf& d, const void* src, size_t bytes) {
    if (d.bytes < bytes) {
        if (d.p) cudaFree(d.p);
        d.p = nullptr;
        d.bytes = 0;
        if (cudaMalloc(&d.p, bytes) != cudaSuccess) return berr(b, SVH_ERR_OOM, "svh_batch_matvec: device allocation failed");
        d.bytes = bytes;
    }
    if (src && cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return berr(b, SVH_ERR_CUDA, "svh_batch_matvec: upload failed");
    return SVH_OK;
}

static FftPlan dev_plan(const FftPlanHost& p) {
    FftPlan d{};
    d.N = p.N;
    d.nst = (int)p.R.size();
    for (int i = 0; i < d.nst && i < MAX_STAGES; ++i) d.R[i] = p.R[i];
    return d;
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

// mode 1: every structure's product on its lane (per-right-hand-side frequencies from the
// batch's device copy), forked from and joined to the batch stream
static int launch_chains(Batch* b, const int32_t* nbs, const void* const* x_dev, void* const* y_dev, int precision,
                         std::string& msg) {
    const size_t n = b->items.size(), L = std::min(b->lanes.size(), n);
    if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return SVH_ERR_CUDA;
    for (size_t l = 0; l < L; ++l)
        if (cudaStreamWaitEvent(b->lanes[l], b->fork, 0) != cudaSuccess) return SVH_ERR_CUDA;
    int rc = SVH_OK;
    size_t off = 0;
    for (size_t i = 0; i < n && rc == SVH_OK; ++i) {
        Handle* h = b->items[i];
        cudaStream_t saved = h->stream;
        h->stream = b->lanes[i % L];
        const double* om = static_cast<const double*>(b->d_omegas.p) + off;
        const double om0 = b->key_om.empty() ? 1.0 : b->key_om[off];
        rc = precision == SVH_FP32 ? launch_matvec32(h, om0, nbs[i], x_dev[i], y_dev[i], 0, om)
                                   : launch_matvec64(h, om0, nbs[i], x_dev[i], y_dev[i], 0, om);
        if (rc) msg = h->err;
        h->stream = saved;
        off += (size_t)nbs[i];
    }
    for (size_t l = 0; l < L; ++l) {
        cudaEventRecord(b->lane_done[l], b->lanes[l]);
        cudaStreamWaitEvent(b->stream, b->lane_done[l], 0);
    }
    return rc;
}

// Builds the queue of one argument set: per-structure descriptors (growing each handle's
// intermediate grids to its right-hand-side count), segments in queue order, counters.
static int build_queue(Batch* b, const int32_t* nbs, const double* const* omegas, const void* const* x_dev,
                       void* const* y_dev, int precision) {
    const int n = (int)b->items.size();
    std::vector<BItem> its(n);
    std::vector<double> oms;
    std::vector<size_t> om_off(n);
    for (int i = 0; i < n; ++i) {
        om_off[i] = oms.size();
        oms.insert(oms.end(), omegas[i], omegas[i] + nbs[i]);
    }
    int rc = bupload(b, b->d_omegas, oms.data(), oms.size() * sizeof(double));
    if (rc) return rc;
    const bool f32 = precision == SVH_FP32;
    const double mu0 = 4e-7 * 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        Handle* h = b->items[i];
        size_t b1, b2;
        matvec_scratch_bytes(h, nbs[i], precision, &b1, &b2);
        if (h->d_B1.bytes < b1 && (rc = dev_alloc(h, h->d_B1, b1))) return berr(b, rc, h->err);
        if (h->d_B2.bytes < b2 && (rc = dev_alloc(h, h->d_B2, b2))) return berr(b, rc, h->err);
        BItem& it = its[i];
        std::memset(&it, 0, sizeof(BItem));
        it.x = x_dev[i];
        it.y = y_dev[i];
        it.B1 = h->d_B1.p;
        it.B2 = h->d_B2.p;
        it.spec = f32 ? h->d_spec32.p : h->d_spec64.p;
        for (int a = 0; a < 3; ++a) it.tw[a] = f32 ? h->d_tw32[a].p : h->d_tw64[a].p;
        it.vidx = static_cast<const int32_t*>(h->d_vidx.p);
        it.rows = static_cast<const int32_t*>(h->d_rows.p);
        it.rowmask = static_cast<const uint8_t*>(h->d_rowmask.p);
        it.zlist = static_cast<const int32_t*>(h->d_zlist.p);
        it.node = static_cast<const int32_t*>(h->d_node.p);
        it.ninc = static_cast<const int32_t*>(h->d_ninc.p);
        it.lam = static_cast<const double*>(h->d_lam.p);
        it.sig0 = static_cast<const double*>(h->d_sig0.p);
        it.omegas = static_cast<const double*>(b->d_omegas.p) + om_off[i];
        it.K = h->K;
        it.M = h->M;
        it.Nvec = 5 * h->K + h->M;
        it.nb = nbs[i];
        it.nza = (int)h->zlist.size();
        it.nrows = (int)h->rows.size();
        it.Kx = h->Kx; it.Ky = h->Ky; it.Kz = h->Kz;
        it.Px = h->Px; it.Py = h->Py;
        it.Hx = h->Hx; it.Hy = h->Hy; it.Hz = h->Hz;
        it.mu = mu0;
        it.dx = h->dx;
        it.inv_P = 1.0 / ((double)h->Px * h->Py * h->Pz);
        it.px = dev_plan(h->plan[0]);
        it.py = dev_plan(h->plan[1]);
        it.pz = dev_plan(h->plan[2]);
        batch_item_shape(it, precision);
        if (!batch_fits(it, precision))
            return berr(b, SVH_ERR_ARG, "svh_batch_matvec: item " + std::to_string(i) + " has FFT sizes above the "
                                        "per-tile limit of the batch kernel");
    }
    // queue order: phase by phase; within a phase the structures with the most work first
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int64_t> work(n, 0);
    for (int i = 0; i < n; ++i)
        for (int p = 0; p < kBatchPhases; ++p) work[i] += its[i].ntile[p];
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
    const int nseg = n * kBatchPhases;
    std::vector<int64_t> seg(nseg + 1, 0);
    std::vector<int> segpi(2 * (size_t)nseg);
    int k = 0;
    for (int p = 0; p < kBatchPhases; ++p)
        for (int i : order) {
            seg[k + 1] = seg[k] + its[i].ntile[p];
            segpi[k] = p;
            segpi[nseg + k] = i;
            ++k;
        }
    if (seg[nseg] >= ((int64_t)1 << 31)) return berr(b, SVH_ERR_ARG, "svh_batch_matvec: batch too large for one queue");
    size_t smem = 0;
    for (const BItem& it : its) smem = std::max(smem, it.smem);
    int32_t zero = 0;
    if ((rc = bupload(b, b->d_items, its.data(), its.size() * sizeof(BItem))) ||
        (rc = bupload(b, b->d_seg, seg.data(), seg.size() * sizeof(int64_t))) ||
        (rc = bupload(b, b->d_segpi, segpi.data(), segpi.size() * sizeof(int))) ||
        (rc = bupload(b, b->d_cnt, nullptr, sizeof(int) * (1 + (size_t)nseg))))
        return rc;
    if (!b->d_status.p && (rc = bupload(b, b->d_status, &zero, sizeof(int)))) return rc;
    if ((rc = batch_queue_grid(precision, smem, b->device, &b->grid)))
        return berr(b, rc, "svh_batch_matvec: kernel attributes could not be set");
    BQueue& q = b->q;
    q.items = static_cast<const BItem*>(b->d_items.p);
    q.nitems = n;
    q.seg_start = static_cast<const int64_t*>(b->d_seg.p);
    q.seg_phase = static_cast<const int*>(b->d_segpi.p);
    q.seg_item = static_cast<const int*>(b->d_segpi.p) + nseg;
    q.nseg = nseg;
    q.counter = static_cast<int*>(b->d_cnt.p);
    q.done = q.counter + 1;
    q.status = static_cast<int*>(b->d_status.p);
    q.wait_ns = (unsigned long long)(b->wait_ms * 1e6);
    q.hold_item = b->hold_item;
    q.hold_phase = b->hold_phase;
    b->smem = smem;
    return SVH_OK;
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
    for (DevBuf* d : {&b->d_items, &b->d_seg, &b->d_segpi, &b->d_cnt, &b->d_status, &b->d_omegas})
        if (d->p) cudaFree(d->p);
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

int svh_batch_set_wait(svh_batch* bb, double limit_ms, int hold_item, int hold_phase) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return SVH_ERR_ARG;
    if (!(limit_ms > 0) || !(limit_ms <= 60000.0) || hold_item < -1 || hold_phase < -1 ||
        hold_phase >= kBatchPhases || (hold_item >= 0) != (hold_phase >= 0))
        return berr(b, SVH_ERR_ARG, "svh_batch_set_wait: bad limit or hold");
    b->wait_ms = limit_ms;
    b->hold_item = hold_item;
    b->hold_phase = hold_phase;
    b->drop_graph();
    return SVH_OK;
}

int svh_batch_set_mode(svh_batch* bb, int mode) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return SVH_ERR_ARG;
    if (mode != 0 && mode != 1) return berr(b, SVH_ERR_ARG, "svh_batch_set_mode: mode must be 0 or 1");
    b->mode = mode;
    b->drop_graph();
    return SVH_OK;
}

int svh_batch_get_mode(const svh_batch* bb) {
    const Batch* b = reinterpret_cast<const Batch*>(bb);
    return b ? b->mode : -1;
}

int svh_batch_autotune(svh_batch* bb, const int32_t* nbs, const double* const* omegas, const void* const* x_dev,
                       void* const* y_dev, int precision, double* ms) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return SVH_ERR_ARG;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaSetDevice(b->device) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        return berr(b, SVH_ERR_CUDA, "svh_batch_autotune: event set-up failed");
    float t[2] = {0, 0};
    int rc = SVH_OK;
    for (int m = 0; m < 2 && !rc; ++m) {
        b->mode = m;
        rc = svh_batch_matvec(bb, nbs, omegas, x_dev, y_dev, precision);   // capture + first launch
        if (!rc) rc = svh_batch_sync(bb);
        if (rc) break;
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < 3 && !rc; ++r) rc = svh_batch_matvec(bb, nbs, omegas, x_dev, y_dev, precision);
        cudaEventRecord(e1, b->stream);
        if (!rc) rc = svh_batch_sync(bb);
        if (!rc) cudaEventElapsedTime(&t[m], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->mode = t[1] < t[0] ? 1 : 0;
    b->drop_graph();
    if (ms) { ms[0] = t[0] / 3; ms[1] = t[1] / 3; }
    return SVH_OK;
}

int svh_batch_matvec(svh_batch* bb, const int32_t* nbs, const double* const* omegas, const void* const* x_dev,
                     void* const* y_dev, int precision) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || !nbs || !omegas || !x_dev || !y_dev || (precision != SVH_FP32 && precision != SVH_FP64))
        return b ? berr(b, SVH_ERR_ARG, "svh_batch_matvec: bad arguments") : SVH_ERR_ARG;
    if (b->items.empty()) return berr(b, SVH_ERR_STATE, "svh_batch_matvec: empty batch");
    if (cudaSetDevice(b->device) != cudaSuccess) return berr(b, SVH_ERR_CUDA, "cudaSetDevice failed");
    const size_t n = b->items.size();
    std::vector<double> om_flat;
    for (size_t i = 0; i < n; ++i) {
        if (nbs[i] <= 0 || !omegas[i] || !x_dev[i] || !y_dev[i])
            return berr(b, SVH_ERR_ARG, "svh_batch_matvec: bad item arguments");
        for (int r = 0; r < nbs[i]; ++r) {
            if (!(omegas[i][r] > 0) || !std::isfinite(omegas[i][r]))
                return berr(b, SVH_ERR_ARG, "svh_batch_matvec: omega must be > 0");
            om_flat.push_back(omegas[i][r]);
        }
        const size_t bytes = (size_t)nbs[i] * (5 * b->items[i]->K + b->items[i]->M) * (precision == SVH_FP32 ? 8 : 16);
        const char* xc = static_cast<const char*>(x_dev[i]);
        const char* yc = static_cast<char*>(y_dev[i]);
        if (xc < yc + bytes && yc < xc + bytes) return berr(b, SVH_ERR_ARG, "svh_batch_matvec: x and y overlap");
    }
    const bool same = b->exec && b->key_prec == precision && b->key_mode == b->mode && b->key_x.size() == n &&
                      std::equal(b->key_x.begin(), b->key_x.end(), x_dev) &&
                      std::equal(b->key_y.begin(), b->key_y.end(), y_dev) &&
                      std::equal(b->key_nb.begin(), b->key_nb.end(), nbs) && b->key_om == om_flat;
    if (!same) {
        b->drop_graph();
        int rc = build_queue(b, nbs, omegas, x_dev, y_dev, precision);
        if (rc) return rc;
        b->key_om = om_flat;
        std::string msg;
        if (b->mode == 1) {
            // run once eagerly so that every buffer a product needs exists before capture
            if (!ensure_lanes(b)) return berr(b, SVH_ERR_CUDA, "svh_batch_matvec: stream set-up failed");
            if ((rc = launch_chains(b, nbs, x_dev, y_dev, precision, msg)))
                return berr(b, rc, "svh_batch_matvec: item product failed: " + msg);
        }
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return berr(b, SVH_ERR_CUDA, "svh_batch_matvec: set-up failed");
        cudaError_t e = cudaStreamBeginCapture(b->stream, b->mode == 1 ? cudaStreamCaptureModeRelaxed
                                                                        : cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = b->mode == 1 ? launch_chains(b, nbs, x_dev, y_dev, precision, msg)
                              : batch_queue_launch(b->q, precision, b->smem, b->grid, b->stream);
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
        b->key_nb.assign(nbs, nbs + n);
        b->key_prec = precision;
        b->key_mode = b->mode;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return berr(b, SVH_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return SVH_OK;
}

int svh_batch_sync(svh_batch* bb) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return SVH_ERR_ARG;
    cudaSetDevice(b->device);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return berr(b, SVH_ERR_CUDA, "svh_batch_sync: stream failed");
    if (!b->d_status.p) return SVH_OK;
    int32_t st = 0;
    if (cudaMemcpy(&st, b->d_status.p, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return berr(b, SVH_ERR_CUDA, "svh_batch_sync: status read failed");
    if (st & SVH_STATUS_QUEUE_TIMEOUT) {
        const int32_t zero = 0;
        cudaMemcpy(b->d_status.p, &zero, 4, cudaMemcpyHostToDevice);
        return berr(b, SVH_ERR_TIMEOUT, "svh_batch_sync: a wait of the batch queue for a pass ran out "
                                        "(the products of this launch are incomplete)");
    }
    return SVH_OK;
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
