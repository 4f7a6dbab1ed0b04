// Instantiation of the MLEM passes for one lane capacity TSP_LMAX (each
// capacity is compiled in its own translation unit).
#include "tsp_launch.h"
#include "tsp_mlem.cuh"

#ifndef TSP_LMAX
#error "define TSP_LMAX before including this file"
#endif

namespace tsp {

namespace {

template <int LMAX, int MODE>
cudaError_t run_pass(const PassArgs& a, cudaStream_t st)
{
    if (a.n_items > 0)
        k_tiles<LMAX, MODE><<<a.grid, kThreads, a.smem, st>>>(a.g, a.tl, a.evs, a.items, a.n_items,
                                                              a.rhop, a.A, a.accum, a.G, a.nseg);
    if (a.outlier_count > 0) {
        const int per_block = kWarps / a.G;
        int blocks = (a.outlier_count + per_block - 1) / per_block;
        if (blocks > a.grid) blocks = a.grid;
        k_outliers<LMAX, MODE><<<blocks, kThreads, 0, st>>>(a.g, a.evs, a.outlier_first,
                                                            a.outlier_count, a.rhop, a.A, a.accum,
                                                            a.G, a.nseg);
    }
    return cudaGetLastError();
}

template <int LMAX, int MODE>
cudaError_t set_smem(size_t smem)
{
    return cudaFuncSetAttribute(k_tiles<LMAX, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

}  // namespace

template <>
cudaError_t launch_pass_l<TSP_LMAX>(int mode, const PassArgs& a, cudaStream_t st)
{
    switch (mode) {
    case kMlem: return run_pass<TSP_LMAX, kMlem>(a, st);
    case kLoglik: return run_pass<TSP_LMAX, kLoglik>(a, st);
    case kGrad: return run_pass<TSP_LMAX, kGrad>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t prepare_pass_l<TSP_LMAX>(int mode, size_t smem)
{
    switch (mode) {
    case kMlem: return set_smem<TSP_LMAX, kMlem>(smem);
    case kLoglik: return set_smem<TSP_LMAX, kLoglik>(smem);
    case kGrad: return set_smem<TSP_LMAX, kGrad>(smem);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tsp
