/*
 * synth_dev.cu -- device side of the seeded input generator (see
 * synth_common.h).  Evaluates exactly the host generator's voxel function on
 * the GPU (bit-identical: every float step is an _rn intrinsic), so that
 * multi-GiB volumes can be produced without a host round trip.  Input
 * generation only: nothing here belongs to the renderer.
 */
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#include "synth_common.h"

struct sy_dev {
    sy_view v; /* pointers refer to device memory */
    sy_nucleus* d_nuclei;
    int64_t* d_cell_start;
    int32_t* d_cell_idx;
};

__global__ void sy_generate_kernel(sy_view v, int64_t x0, int64_t nx, int64_t y0, int64_t ny, int64_t z0, int64_t nz,
                                   uint16_t* __restrict__ out) {
    int64_t total = nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % nx, r = i / nx;
        int64_t y = r % ny, z = r / ny;
        uint16_t vals[SY_MAXC];
        sy_voxel(&v, x0 + x, y0 + y, z0 + z, vals);
        for (int c = 0; c < v.C; ++c) out[i * v.C + c] = vals[c];
    }
}

extern "C" {

/* Copies a host specification (its sy_view) to the current device. Returns NULL on failure. */
void* sy_dev_create(const sy_view* hv, int64_t n_nuclei, int64_t n_cells, int64_t n_idx) {
    sy_dev* d = (sy_dev*)calloc(1, sizeof(sy_dev));
    d->v = *hv;
    size_t bn = sizeof(sy_nucleus) * (size_t)(n_nuclei > 0 ? n_nuclei : 1);
    size_t bs = sizeof(int64_t) * (size_t)(n_cells + 1);
    size_t bi = sizeof(int32_t) * (size_t)(n_idx > 0 ? n_idx : 1);
    if (cudaMalloc(&d->d_nuclei, bn) != cudaSuccess || cudaMalloc(&d->d_cell_start, bs) != cudaSuccess ||
        cudaMalloc(&d->d_cell_idx, bi) != cudaSuccess) {
        cudaFree(d->d_nuclei);
        cudaFree(d->d_cell_start);
        cudaFree(d->d_cell_idx);
        free(d);
        return nullptr;
    }
    cudaMemcpy(d->d_nuclei, hv->nuclei, sizeof(sy_nucleus) * (size_t)n_nuclei, cudaMemcpyHostToDevice);
    cudaMemcpy(d->d_cell_start, hv->cell_start, bs, cudaMemcpyHostToDevice);
    if (n_idx > 0) cudaMemcpy(d->d_cell_idx, hv->cell_idx, sizeof(int32_t) * (size_t)n_idx, cudaMemcpyHostToDevice);
    d->v.nuclei = d->d_nuclei;
    d->v.cell_start = d->d_cell_start;
    d->v.cell_idx = d->d_cell_idx;
    return d;
}

void sy_dev_destroy(void* h) {
    sy_dev* d = (sy_dev*)h;
    if (!d) return;
    cudaFree(d->d_nuclei);
    cudaFree(d->d_cell_start);
    cudaFree(d->d_cell_idx);
    free(d);
}

/* Box [x0,x1) x [y0,y1) x [z0,z1) -> out[z][y][x][C] (device pointer), stream-ordered. */
int sy_dev_generate_box(void* h, int64_t x0, int64_t x1, int64_t y0, int64_t y1, int64_t z0, int64_t z1, uint16_t* out,
                        void* stream) {
    sy_dev* d = (sy_dev*)h;
    if (!d || x0 < 0 || y0 < 0 || z0 < 0 || x1 > d->v.X || y1 > d->v.Y || z1 > d->v.Z || x1 < x0 || y1 < y0 || z1 < z0)
        return -1;
    int64_t total = (x1 - x0) * (y1 - y0) * (z1 - z0);
    if (total == 0) return 0;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 148 * 64) blocks = 148 * 64;
    sy_generate_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d->v, x0, x1 - x0, y0, y1 - y0, z0, z1 - z0,
                                                                          out);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
}
