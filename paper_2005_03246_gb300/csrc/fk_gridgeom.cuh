// fk_gridgeom.cuh -- rectilinear grid geometry shared by the grid ECDF
// (fk_grid.cu) and the grid KDE (fk_kgrid.cu): axis descriptors, the exact
// binning of eq. (partial sums) and the per-axis set-up kernel.
#pragma once

#include "fk_internal.cuh"

namespace fk {

struct AxisInfo {
    int uniform;
    double z0, inv_dz;
};

struct GridGeom {
    int d;
    int64_t M[8];                 // axis lengths
    const double* z[8];           // device pointer to axis k values
    const AxisInfo* info;         // device, [d]
};


// bin index j in [0, M]: number of axis values strictly below v, i.e.
// z_{j-1} < v <= z_j with z_{-1} = -inf, z_M = +inf (eq. partial sums).
__device__ __forceinline__ int64_t bin_of(double v, const double* __restrict__ z, int64_t M,
                                          int uniform, double z0, double inv_dz) {
    if (uniform) {
        // Algorithm 7: 1 + ceil((x - z_1)/dz) in 1-based indexing, then an exact fix-up.
        double g = ceil((v - z0) * inv_dz);
        int64_t j = (g <= 0.0) ? 0 : (g >= (double)M ? M : (int64_t)g);
        for (int it = 0; it < 4; ++it) {
            if (j > 0 && !(z[j - 1] < v)) { --j; continue; }
            if (j < M && !(v <= z[j])) { ++j; continue; }
            return j;
        }
    }
    int64_t lo = 0, hi = M;   // binary search (Algorithm 6 equivalent)
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (z[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}


// Per-axis set-up: strict monotonicity check (eq. partial sums needs
// z_{k,1} < ... < z_{k,M_k}) and detection of uniform spacing (Algorithm 7).
static __global__ void k_axis_setup(GridGeom g, AxisInfo* __restrict__ info, int* __restrict__ err) {
    int k = blockIdx.x;
    if (k >= g.d) return;
    const double* z = g.z[k];
    int64_t M = g.M[k];
    __shared__ int bad, nonuni;
    if (threadIdx.x == 0) { bad = 0; nonuni = 0; }
    __syncthreads();
    double z0 = z[0];
    double dz = M > 1 ? (z[M - 1] - z0) / (double)(M - 1) : 1.0;
    for (int64_t j = threadIdx.x; j < M; j += blockDim.x) {
        double v = z[j];
        if (!(v == v) || (j > 0 && !(z[j - 1] < v))) bad = 1;
        if (fabs(v - (z0 + (double)j * dz)) > 1e-6 * fabs(dz)) nonuni = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bad) atomicCAS(err, 0, (int)DEV_AXIS);
        info[k].uniform = (M > 1 && !nonuni && dz > 0.0) ? 1 : 0;
        info[k].z0 = z0;
        info[k].inv_dz = (dz > 0.0) ? 1.0 / dz : 0.0;
    }
}

}  // namespace fk
