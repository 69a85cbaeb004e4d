// bs_vel_f32_q4.cu -- float32 instances of the velocity kernel for the four-point far rule (the
// workhorse, and the widest choice for the autotuner): points per thread, tile, stages, register
// budget, near pairs (drained in the kernel: routine called, inlined, or inlined with its state in shared
// memory; or left to the near pass), ray bundle, the far sweep's register pairing, and the unroll of its
// tet loop.
#include "bs_velocity_kernel.cuh"

namespace bs {
namespace {

#define BS_V(P, TILE, S, MINB, DR, U, PK, UJ) \
    { {P, TILE, S, MINB, DR, U, PK, UJ}, &launch_t<float, 4, P, 128, TILE, S, MINB, DR, false, U, PK, UJ> }

// variant 0 is the default; the first variant with one point per thread and tiles of 32 serves small meshes
const VariantEntry kF32Q4[] = {
    // near pairs left to the near pass: the far sweep has no drain (no spills at 4 CTAs per SM); variant 0 unrolls
    // the tet loop by 4 (the default for sizes the autotuner has not seen)
    BS_V(3, 32, 2, 4, 3, 1, false, 4), BS_V(3, 32, 2, 4, 3, 1, false, 1), BS_V(3, 64, 2, 4, 3, 1, false, 1),
    BS_V(4, 32, 2, 4, 3, 1, false, 1),
    // one point per thread (small meshes)
    BS_V(1, 32, 4, 5, 0, 1, false, 1),
    BS_V(2, 32, 2, 4, 3, 1, false, 2), BS_V(4, 32, 2, 4, 3, 1, true, 1), BS_V(3, 32, 2, 4, 3, 1, false, 2),
    // near pairs drained in the far kernel: the pair's state in shared memory
    BS_V(3, 32, 2, 4, 2, 1, false, 1), BS_V(4, 32, 2, 4, 2, 1, false, 1),
    // ray bundles of 2 and 4 lines per lane
    BS_V(1, 32, 4, 5, 0, 2, false, 1), BS_V(1, 32, 4, 5, 0, 4, false, 1),
    // near routine in registers, inlined or called
    BS_V(3, 32, 2, 4, 1, 1, false, 1), BS_V(3, 64, 2, 4, 1, 1, false, 1), BS_V(2, 64, 2, 4, 1, 1, false, 1),
    BS_V(3, 32, 3, 4, 1, 1, false, 1), BS_V(3, 16, 3, 4, 1, 1, false, 1), BS_V(2, 32, 4, 3, 1, 1, false, 1),
    BS_V(2, 32, 3, 4, 0, 1, false, 1), BS_V(2, 32, 4, 5, 1, 1, false, 1), BS_V(3, 32, 2, 4, 1, 4, false, 1),
    BS_V(4, 32, 2, 3, 1, 1, true, 1), BS_V(1, 32, 4, 5, 2, 1, false, 1),
    // one point per thread with the near pairs left to the near pass (small meshes, batches)
    BS_V(1, 32, 3, 7, 3, 1, false, 2), BS_V(1, 32, 4, 6, 3, 1, false, 2), BS_V(2, 32, 3, 5, 3, 1, false, 2),
    // three stages, the tet loop unrolled by 2; three stages unrolled by 4
    BS_V(3, 32, 3, 4, 3, 1, false, 2), BS_V(3, 32, 3, 4, 3, 1, false, 4),
};
#undef BS_V

}  // namespace

VariantList variants_f32_q4() { return {kF32Q4, (int)(sizeof(kF32Q4) / sizeof(kF32Q4[0]))}; }

}  // namespace bs
