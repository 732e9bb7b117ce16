// Fused-pass kernels instantiated for float storage (one translation unit per
// precision so the two compile in parallel).
#include "tl_pass_impl.cuh"

namespace tl {

cudaError_t launch_pass_f32(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                             double *slots, bool measure_only, cudaStream_t s, const TmaMaps *maps)
{
    switch (m.nf) {
    case 1: return launch_t<float, 1>(m, fp, c, g, sc, slots, measure_only, s, maps);
    case 2: return launch_t<float, 2>(m, fp, c, g, sc, slots, measure_only, s, maps);
    case 3: return launch_t<float, 3>(m, fp, c, g, sc, slots, measure_only, s, maps);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_group_f32(int nf, const BatchJob *jobs, const unsigned *first_item, int njobs, unsigned total,
                              const PassCoef &c, int grid, cudaStream_t s)
{
    // the staged job table (see fused_pass_group)
    const size_t smem = njobs <= kGroupStagedJobs ? (size_t)njobs * sizeof(unsigned) : 0;
    switch (nf) {
    case 1: fused_pass_group<float, 1><<<grid, 256, smem, s>>>(jobs, first_item, njobs, total, c); break;
    case 2: fused_pass_group<float, 2><<<grid, 256, smem, s>>>(jobs, first_item, njobs, total, c); break;
    case 3: fused_pass_group<float, 3><<<grid, 256, smem, s>>>(jobs, first_item, njobs, total, c); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tl
