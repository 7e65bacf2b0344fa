// od_tiles.cu -- instantiates the tile kernels for one arithmetic mode and
// one stencil.  Built once per (mode, stencil) with -DOD_AMODE=<0..15> and
// -DOD_STENCIL=<0 (3D 7-point) | 1 (2D 5-point)> (the build compiles the
// copies in parallel); od_kernels.cu dispatches on both at launch time.
#include "od_tile.cuh"

#ifndef OD_AMODE
#error "compile with -DOD_AMODE=<mode>"
#endif
#ifndef OD_STENCIL
#define OD_STENCIL 0
#endif
#if OD_STENCIL == 0
#define OD_TILE_FN OD_CAT(tile_kernel_am, OD_AMODE)
#else
#define OD_TILE_FN OD_CAT(tile_kernel2d_am, OD_AMODE)
#endif

#define OD_CAT2(a, b) a##b
#define OD_CAT(a, b) OD_CAT2(a, b)

namespace od {

// kind 0: k_tiles (per-chare compute), 1: k_tiles (fused step), 2:
// k_persistent, 3: k_tiles_multi, 4: k_persistent_multi
void *OD_TILE_FN(int threads, int cpt, int kind) {
    using namespace tile;
#define OD_CASE(NT_, C_)                                                          \
    if (threads == NT_ && cpt == C_) {                                            \
        if (kind == 0) return (void *)k_tiles<NT_, C_, false, OD_AMODE, OD_STENCIL>; \
        if (kind == 1) return (void *)k_tiles<NT_, C_, true, OD_AMODE, OD_STENCIL>;  \
        if (kind == 3) return (void *)k_tiles_multi<NT_, C_, OD_AMODE, OD_STENCIL>;  \
        if (kind == 4) return (void *)k_persistent_multi<NT_, C_, OD_AMODE, OD_STENCIL>; \
        return (void *)k_persistent<NT_, C_, OD_AMODE, OD_STENCIL>;                  \
    }
    OD_CASE(128, 2) OD_CASE(128, 4) OD_CASE(128, 8)
    OD_CASE(256, 1) OD_CASE(256, 2) OD_CASE(256, 4) OD_CASE(256, 8)
    OD_CASE(512, 1) OD_CASE(512, 2)
#undef OD_CASE
    return nullptr;
}

}  // namespace od
