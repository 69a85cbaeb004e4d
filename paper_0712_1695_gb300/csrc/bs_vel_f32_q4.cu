// bs_vel_f32_q4.cu -- float32 instances of the velocity kernel for the four-point far rule (the
// workhorse, and the widest choice for the autotuner): points per thread, tile, stages, register
// budget, near routine inlined or called, ray bundle, and the far sweep's register pairing.
#include "bs_velocity_kernel.cuh"

namespace bs {
namespace {

#define BS_V(P, TILE, S, MINB, INL, U, PK) \
    { {P, TILE, S, MINB, INL, U, PK}, &launch_t<float, 4, P, 128, TILE, S, MINB, INL, false, U, PK> }

// variant 0 is the default; variant 4 (one point per thread) serves small meshes
const VariantEntry kF32Q4[] = {
    BS_V(3, 32, 2, 4, true, 1, false),  BS_V(2, 32, 4, 3, false, 1, false), BS_V(4, 32, 4, 2, false, 1, false),
    BS_V(2, 32, 2, 4, false, 1, false), BS_V(1, 32, 4, 5, false, 1, false), BS_V(2, 32, 3, 4, false, 1, false),
    BS_V(2, 32, 4, 3, true, 1, false),  BS_V(3, 32, 3, 4, true, 1, false),  BS_V(2, 32, 4, 5, true, 1, false),
    BS_V(2, 32, 3, 4, true, 1, false),  BS_V(4, 32, 3, 3, true, 1, false),  BS_V(3, 32, 3, 4, false, 1, false),
    // tiles of 64 and 16 tets
    BS_V(3, 64, 2, 4, true, 1, false),  BS_V(3, 16, 3, 4, true, 1, false),  BS_V(2, 64, 2, 4, true, 1, false),
    BS_V(1, 16, 4, 5, false, 1, false),
    // ray bundles of 2 and 4 lines per lane
    BS_V(1, 32, 4, 5, false, 2, false), BS_V(1, 32, 4, 5, false, 4, false), BS_V(3, 32, 2, 4, true, 4, false),
    // point-pair far sweep
    BS_V(4, 32, 2, 4, true, 1, true),   BS_V(4, 64, 2, 4, true, 1, true),   BS_V(6, 32, 2, 3, true, 1, true),
    BS_V(2, 32, 2, 5, true, 1, true),   BS_V(4, 32, 2, 3, true, 1, true),
};
#undef BS_V

}  // namespace

VariantList variants_f32_q4() { return {kF32Q4, (int)(sizeof(kF32Q4) / sizeof(kF32Q4[0]))}; }

}  // namespace bs
