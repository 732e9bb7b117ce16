// Fused-pass kernels instantiated for float storage (one translation unit per
// precision so the two compile in parallel).
#include "tl_pass_impl.cuh"

namespace tl {

cudaError_t launch_pass_f32(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                             double *slots, bool measure_only, cudaStream_t s)
{
    switch (m.nf) {
    case 1: return launch_t<float, 1>(m, fp, c, g, sc, slots, measure_only, s);
    case 2: return launch_t<float, 2>(m, fp, c, g, sc, slots, measure_only, s);
    case 3: return launch_t<float, 3>(m, fp, c, g, sc, slots, measure_only, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace tl
