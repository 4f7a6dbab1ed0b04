// Instantiation of the MLEM passes for one lane capacity TSP_LMAX (each
// capacity is compiled in its own translation unit), for one lane per image
// row (nseg = 1) and for two lanes per row (nseg = 2).
#include "tsp_launch.h"
#include "tsp_mlem.cuh"

#ifndef TSP_LMAX
#error "define TSP_LMAX before including this file"
#endif

namespace tsp {

namespace {

template <int LMAX, int MODE, int NSEG>
cudaError_t run_pass(const PassArgs& a, cudaStream_t st)
{
    if (a.n_items > 0)
        k_tiles<LMAX, MODE, NSEG><<<a.grid, kThreads, a.smem, st>>>(
            a.g, a.tl, a.evs, a.items, a.n_items, a.rhop, a.A, a.accum, a.G);
    if (a.outlier_count > 0) {
        const int per_block = kWarps / a.G;
        int blocks = (a.outlier_count + per_block - 1) / per_block;
        if (blocks > a.grid) blocks = a.grid;
        k_outliers<LMAX, MODE, NSEG><<<blocks, kThreads, 0, st>>>(
            a.g, a.evs, a.outlier_first, a.outlier_count, a.rhop, a.A, a.accum, a.G);
    }
    return cudaGetLastError();
}

template <int LMAX, int MODE, int NSEG>
cudaError_t set_smem(size_t smem)
{
    return cudaFuncSetAttribute(k_tiles<LMAX, MODE, NSEG>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int LMAX, int NSEG>
cudaError_t run_mode(int mode, const PassArgs& a, cudaStream_t st)
{
    switch (mode) {
    case kMlem: return run_pass<LMAX, kMlem, NSEG>(a, st);
    case kLoglik: return run_pass<LMAX, kLoglik, NSEG>(a, st);
    case kGrad: return run_pass<LMAX, kGrad, NSEG>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int LMAX, int NSEG>
cudaError_t smem_mode(int mode, size_t smem)
{
    switch (mode) {
    case kMlem: return set_smem<LMAX, kMlem, NSEG>(smem);
    case kLoglik: return set_smem<LMAX, kLoglik, NSEG>(smem);
    case kGrad: return set_smem<LMAX, kGrad, NSEG>(smem);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <>
cudaError_t launch_pass_l<TSP_LMAX>(int mode, const PassArgs& a, cudaStream_t st)
{
    return a.nseg == 1 ? run_mode<TSP_LMAX, 1>(mode, a, st) : run_mode<TSP_LMAX, 2>(mode, a, st);
}

template <>
cudaError_t prepare_pass_l<TSP_LMAX>(int mode, size_t smem)
{
    cudaError_t e = smem_mode<TSP_LMAX, 1>(mode, smem);
    if (e == cudaSuccess) e = smem_mode<TSP_LMAX, 2>(mode, smem);
    return e;
}

}  // namespace tsp
