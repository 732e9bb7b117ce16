// Fused-pass kernels instantiated for double storage (one translation unit per
// precision so the two compile in parallel).
#include "tl_pass_impl.cuh"

namespace tl {

cudaError_t launch_pass_f64(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                             double *slots, bool measure_only, cudaStream_t s, const TmaMaps *maps)
{
    switch (m.nf) {
    case 1: return launch_t<double, 1>(m, fp, c, g, sc, slots, measure_only, s, maps);
    case 2: return launch_t<double, 2>(m, fp, c, g, sc, slots, measure_only, s, maps);
    case 3: return launch_t<double, 3>(m, fp, c, g, sc, slots, measure_only, s, maps);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_group_f64(int nf, int variant, int prefetch, int stages, size_t smem, const BatchJob *jobs,
                              const unsigned *first_item, int njobs, unsigned total, const PassCoef &c, int grid,
                              cudaStream_t s)
{
    if (variant == kVariantTma) {
        switch (nf) {
        case 1: return launch_tma_group_t<double, 1>(stages, smem, jobs, first_item, njobs, total, c, s);
        case 2: return launch_tma_group_t<double, 2>(stages, smem, jobs, first_item, njobs, total, c, s);
        case 3: return launch_tma_group_t<double, 3>(stages, smem, jobs, first_item, njobs, total, c, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (nf) {
    case 1: return launch_group_t<double, 1>(prefetch, jobs, first_item, njobs, total, c, grid, s);
    case 2: return launch_group_t<double, 2>(prefetch, jobs, first_item, njobs, total, c, grid, s);
    case 3: return launch_group_t<double, 3>(prefetch, jobs, first_item, njobs, total, c, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace tl
