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

template <int LMAX, int MODE, int NSEG, bool GLD = false>
cudaError_t run_pass(const PassArgs& a, cudaStream_t st)
{
    if (a.n_items > 0) {
        Inst p;
        p.g = a.g;
        p.tl = a.tl;
        p.evs = a.evs;
        p.rhop = a.rhop;
        p.A = a.A;
        p.accum = a.accum;
        p.G = a.G;
        p.pad = 0;
        if (a.g.kz != 0.0f)
            k_tiles<LMAX, MODE, NSEG, false, GLD, true>
                <<<a.grid, pass_threads(LMAX, MODE, NSEG, false), a.smem, st>>>(
                p, nullptr, a.items, a.n_items, &a.accum->queue);
        else
            k_tiles<LMAX, MODE, NSEG, false, GLD, false>
                <<<a.grid, pass_threads(LMAX, MODE, NSEG, false), a.smem, st>>>(
                p, nullptr, a.items, a.n_items, &a.accum->queue);
    }
    if (a.outlier_count > 0) {
        const int per_block = group_count(pass_threads(LMAX, MODE, NSEG, false) / 32, a.G);
        int blocks = (a.outlier_count + per_block - 1) / per_block;
        if (blocks > a.grid) blocks = a.grid;
        k_outliers<LMAX, MODE, NSEG><<<blocks, pass_threads(LMAX, MODE, NSEG, false), 0, st>>>(
            a.g, a.evs, a.outlier_first, a.outlier_count, a.rhop, a.A, a.accum, a.G);
    }
    return cudaGetLastError();
}

template <int LMAX, int MODE, int NSEG, bool GLD, bool KZ>
cudaError_t set_smem_one(size_t smem)
{
    return cudaFuncSetAttribute(k_tiles<LMAX, MODE, NSEG, false, GLD, KZ>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int LMAX, int MODE, int NSEG>
cudaError_t set_smem(size_t smem)
{
    cudaError_t e = set_smem_one<LMAX, MODE, NSEG, false, false>(smem);
    if (e == cudaSuccess) e = set_smem_one<LMAX, MODE, NSEG, false, true>(smem);
    if constexpr (NSEG == 2) {
        if (e == cudaSuccess) e = set_smem_one<LMAX, MODE, NSEG, true, false>(smem);
        if (e == cudaSuccess) e = set_smem_one<LMAX, MODE, NSEG, true, true>(smem);
    }
    return e;
}

// Batched form: one persistent launch over the items of every reconstruction
// (MLEM and gradient passes).
template <int LMAX, int MODE, int NSEG>
cudaError_t run_batch(const BatchArgs& a, cudaStream_t st)
{
    Inst none{};
    if (a.n_items > 0) {
        if (a.kz)
            k_tiles<LMAX, MODE, NSEG, true, false, true>
                <<<a.grid, pass_threads(LMAX, MODE, NSEG, true), a.smem, st>>>(
                    none, a.table, a.items, a.n_items, a.queue);
        else
            k_tiles<LMAX, MODE, NSEG, true, false, false>
                <<<a.grid, pass_threads(LMAX, MODE, NSEG, true), a.smem, st>>>(
                    none, a.table, a.items, a.n_items, a.queue);
    }
    if (a.n_outlier_items > 0)
        k_outliers_batch<LMAX, MODE, NSEG>
            <<<a.n_outlier_items < a.grid ? a.n_outlier_items : a.grid,
               pass_threads(LMAX, MODE, NSEG, true), 0, st>>>(
                a.table, a.outlier_items, a.n_outlier_items);
    return cudaGetLastError();
}

template <int LMAX, int NSEG>
cudaError_t run_batch_mode(int mode, const BatchArgs& a, cudaStream_t st)
{
    switch (mode) {
    case kMlem: return run_batch<LMAX, kMlem, NSEG>(a, st);
    case kGrad: return run_batch<LMAX, kGrad, NSEG>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int LMAX, int NSEG>
cudaError_t batch_smem(size_t smem)
{
    const int v = (int)smem;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_tiles<LMAX, kMlem, NSEG, true, false, false>, at, v);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tiles<LMAX, kMlem, NSEG, true, false, true>, at, v);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tiles<LMAX, kGrad, NSEG, true, false, false>, at, v);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tiles<LMAX, kGrad, NSEG, true, false, true>, at, v);
    return e;
}

template <int LMAX, int NSEG>
cudaError_t run_mode(int mode, const PassArgs& a, cudaStream_t st)
{
    if (NSEG == 2 && a.gld) {
        switch (mode) {
        case kMlem: return run_pass<LMAX, kMlem, 2, true>(a, st);
        case kLoglik: return run_pass<LMAX, kLoglik, 2, true>(a, st);
        case kGrad: return run_pass<LMAX, kGrad, 2, true>(a, st);
        default: return cudaErrorInvalidValue;
        }
    }
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

template <>
cudaError_t launch_batch_pass_l<TSP_LMAX>(int mode, const BatchArgs& a, cudaStream_t st)
{
    return a.nseg == 1 ? run_batch_mode<TSP_LMAX, 1>(mode, a, st)
                       : run_batch_mode<TSP_LMAX, 2>(mode, a, st);
}

template <>
cudaError_t prepare_batch_pass_l<TSP_LMAX>(size_t smem)
{
    cudaError_t e = batch_smem<TSP_LMAX, 1>(smem);
    if (e == cudaSuccess) e = batch_smem<TSP_LMAX, 2>(smem);
    return e;
}

}  // namespace tsp
