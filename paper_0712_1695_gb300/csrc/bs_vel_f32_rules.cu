// bs_vel_f32_rules.cu -- float32 instances of the velocity kernel for the 1-, 8-, 27- and 64-point far
// rules (larger rules take smaller tiles: their far records are longer).
#include "bs_velocity_kernel.cuh"

namespace bs {
namespace {

#define BS_V(Q, P, TILE, S, MINB, DR, U, PK) \
    { {P, TILE, S, MINB, DR, U, PK, 1}, &launch_t<float, Q, P, 128, TILE, S, MINB, DR, false, U, PK, 1> }

// the fifth argument: near pairs drained in the kernel by the routine inlined (1) or called (0), or left
// to the near pass (3)
const VariantEntry kF32Q1[] = {BS_V(1, 2, 32, 4, 4, 1, 1, false), BS_V(1, 1, 32, 4, 5, 0, 1, false),
                               BS_V(1, 4, 32, 2, 4, 1, 1, true), BS_V(1, 2, 32, 4, 4, 1, 1, true),
                               BS_V(1, 4, 32, 2, 4, 3, 1, true)};
const VariantEntry kF32Q8[] = {BS_V(8, 2, 16, 4, 4, 1, 1, false), BS_V(8, 1, 16, 4, 5, 0, 1, false),
                               BS_V(8, 2, 32, 3, 4, 1, 1, false), BS_V(8, 2, 16, 4, 4, 3, 1, false)};
const VariantEntry kF32Q27[] = {BS_V(27, 1, 16, 4, 4, 0, 1, false), BS_V(27, 2, 16, 3, 4, 0, 1, false),
                                BS_V(27, 1, 8, 4, 4, 0, 1, false), BS_V(27, 2, 16, 3, 4, 3, 1, false)};
const VariantEntry kF32Q64[] = {BS_V(64, 1, 8, 4, 4, 0, 1, false), BS_V(64, 2, 8, 3, 4, 0, 1, false),
                                BS_V(64, 1, 16, 2, 4, 0, 1, false), BS_V(64, 2, 8, 3, 4, 3, 1, false)};
#undef BS_V

template <size_t N>
VariantList list(const VariantEntry (&v)[N])
{
    return {v, (int)N};
}

}  // namespace

VariantList variants_f32_rules(int Q)
{
    switch (Q) {
    case 1: return list(kF32Q1);
    case 8: return list(kF32Q8);
    case 27: return list(kF32Q27);
    case 64: return list(kF32Q64);
    default: return {};
    }
}

}  // namespace bs
