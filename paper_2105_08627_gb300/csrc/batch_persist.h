// batch_persist.h -- descriptors of the persistent batch launch (batch_persist.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_plan.h"
#include "svh.h"

namespace svh {

constexpr int kBatchPhases = 6;   // x-fwd, node rows, y-fwd, z pass, y-inv, x-inv + epilogue

// One structure of the batch: its grid, device arrays, right-hand sides and tile shapes.
struct BItem {
    const void* x;            // nb * Nvec complex (float2 or double2), item b at b * Nvec
    void* y;
    void* B1;                 // [nb*5][nza][Ky][Px]
    void* B2;                 // [nb*5][nza][Py][Px]
    const void* spec;         // octant spectra [7][Hz][Hy][Hx] (float or double)
    const void* tw[3];        // exp(-2 pi i m / P_a), m < P_a
    const int32_t* vidx;      // [nza][Ky][Kx] voxel index or -1
    const int32_t* rows;      // active rows zi*Ky + y
    const uint8_t* rowmask;   // [nza][Ky]
    const int32_t* zlist;     // active planes
    const int32_t* node;      // [K][6]
    const int32_t* ninc;      // [M][2] voxel*6+face touching each node, or -1
    const double* lam;
    const double* sig0;
    const double* omegas;     // [nb] angular frequency of each right-hand side
    int64_t K, M, Nvec;
    int nb, nza, nrows, Kx, Ky, Kz, Px, Py, Hx, Hy, Hz;
    double mu, dx, inv_P;
    FftPlan px, py, pz;
    int lpb, tby, tbz;        // x lines, y columns, z columns per tile
    int ntile[kBatchPhases];  // tiles of each phase
    size_t smem;              // dynamic shared memory the largest tile needs
};

// The device work queue: segments (phase, item) in queue order, tile counts, counters.
struct BQueue {
    const BItem* items;
    int nitems;
    const int64_t* seg_start;   // [nseg + 1] first queue index of each segment
    const int* seg_phase;       // [nseg]
    const int* seg_item;        // [nseg]
    int nseg;
    int* counter;               // next queue index; done = counter + 1
    int* done;                  // [nitems][kBatchPhases] completed tiles
    int* status;                // status word (SVH_STATUS_QUEUE_TIMEOUT)
    unsigned long long wait_ns; // bound of each dependency wait
    int hold_item, hold_phase;  // diagnostic: this (item, phase) count is never reached (-1: none)
};

void batch_item_shape(BItem& it, int precision);
bool batch_fits(const BItem& it, int precision);
int batch_queue_grid(int precision, size_t smem, int device, int* grid);
// clears counter and done (one memset) and launches the persistent kernel on s
int batch_queue_launch(const BQueue& q, int precision, size_t smem, int grid, cudaStream_t s);

}  // namespace svh
