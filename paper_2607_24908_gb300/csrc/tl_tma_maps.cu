// Tensor maps of a lattice's arrays for the TMA pass: the driver's
// cuTensorMapEncodeTiled over each padded array (box shape and L2 promotion
// set here).  Kept apart from the rest of the host runtime because, with the
// kernel sources, it fixes the DRAM traffic of the TMA pass.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdlib.h>
#include <string.h>

#include "tl_internal.cuh"
#include "tl_lattice.cuh"

using tl::fail;

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (a function-local static: thread-safe initialisation).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    }();
    return fn;
}

// Encode the tensor maps of both buffer parities for the current tile shape:
// 3-D (padded row, row incl. ghost rows, plane) over each array, boxes
// (txt W + 2W, txt W or W) x (ty + 2) x 1 (TmaMaps).
int encode_maps(tl_lattice *L)
{
    const tl::PassGeom &g = L->geom;
    if (L->maps_txt == g.txt && L->maps_ty == g.ty) return TL_OK;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(TL_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const size_t esz = L->esz;
    const int W = (int)(16 / esz);
    const tl::Layout lay = tl::layout_of(L->N, esz);
    const cuuint64_t dims[3] = {(cuuint64_t)lay.pitch, (cuuint64_t)(L->N + 2), (cuuint64_t)L->N};
    const cuuint64_t strides[2] = {(cuuint64_t)lay.pitch * esz, (cuuint64_t)lay.pplane * esz};
    // Test hook (host-side fault injection): TL_TEST_STALL_TMA encodes boxes one
    // row short, so every stage receives fewer bytes than its barrier expects and
    // the kernel's bounded waits expire (TL_ETIMEOUT) -- a wait that runs out,
    // with every copy inside its stage region.
    const bool stall = getenv("TL_TEST_STALL_TMA") != nullptr;
    const cuuint32_t rows = (cuuint32_t)(g.ty + (stall ? 1 : 2));
    const cuuint32_t boxes[3][3] = {{(cuuint32_t)(g.txt * W + 2 * W), rows, 1u},  // kMapTile
                                    {(cuuint32_t)(g.txt * W), rows, 1u},          // kMapBody
                                    {(cuuint32_t)W, rows, 1u}};                   // kMapSide
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    // L2 promotion of the copies: 64 bytes (measured at N = 256 ... 1024 two
    // fields, 256^3 one field and the grouped ensemble: 0.1-0.5% faster than
    // 256 bytes, 3.4% fewer DRAM reads at 1024^3).  Environment override for
    // tuning experiments: TL_TMA_L2_PROMOTION = none, 64, 128 or 256.
    CUtensorMapL2promotion promo = CU_TENSOR_MAP_L2_PROMOTION_L2_64B;
    if (const char *v = getenv("TL_TMA_L2_PROMOTION")) {
        if (strcmp(v, "none") == 0) promo = CU_TENSOR_MAP_L2_PROMOTION_NONE;
        else if (strcmp(v, "128") == 0) promo = CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
        else if (strcmp(v, "256") == 0) promo = CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
    }
    for (int par = 0; par < 2; ++par)
        for (int k = 0; k < 3; ++k)
            for (int f = 0; f < L->nf; ++f)
                for (int a = 0; a < 2; ++a) {
                    void *base = static_cast<char *>(L->buf[par][a][f]) - lay.origin * esz;
                    CUresult r = enc(&L->maps[par].map[k][2 * f + a],
                                     esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                                     base, dims, strides, boxes[k], estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                     CU_TENSOR_MAP_SWIZZLE_NONE, promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                    if (r != CUDA_SUCCESS) return fail(TL_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
                }
    L->maps_txt = g.txt;
    L->maps_ty = g.ty;
    return TL_OK;
}

}  // namespace

int tl::lattice_tma_maps(tl_lattice *L) { return encode_maps(L); }
