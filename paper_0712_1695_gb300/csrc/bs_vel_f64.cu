// bs_vel_f64.cu -- float64 instances of the velocity kernel (every rule; bound by the float64 pipe).
#include "bs_velocity_kernel.cuh"

namespace bs {
namespace {

// DR: near pairs drained in the kernel (1) or left to the near pass (3)
#define BS_V(Q, P, TILE, S, MINB, DR) \
    { {P, TILE, S, MINB, DR, 1, false, 1}, &launch_t<double, Q, P, 128, TILE, S, MINB, DR, false, 1, false, 1> }

const VariantEntry kF64Q1[] = {BS_V(1, 2, 32, 4, 4, 1), BS_V(1, 1, 32, 4, 4, 1), BS_V(1, 1, 32, 4, 4, 3)};
const VariantEntry kF64Q4[] = {BS_V(4, 1, 32, 2, 4, 1), BS_V(4, 2, 32, 2, 3, 1), BS_V(4, 1, 64, 2, 4, 1),
                               BS_V(4, 1, 16, 3, 4, 1), BS_V(4, 1, 32, 2, 4, 3)};
const VariantEntry kF64Q8[] = {BS_V(8, 2, 16, 4, 4, 1), BS_V(8, 1, 16, 4, 4, 1), BS_V(8, 1, 16, 4, 4, 3)};
const VariantEntry kF64Q27[] = {BS_V(27, 1, 16, 4, 4, 1), BS_V(27, 1, 8, 4, 4, 1), BS_V(27, 1, 16, 4, 4, 3)};
const VariantEntry kF64Q64[] = {BS_V(64, 1, 8, 4, 4, 1), BS_V(64, 1, 4, 4, 4, 1), BS_V(64, 1, 8, 4, 4, 3)};
#undef BS_V

template <size_t N>
VariantList list(const VariantEntry (&v)[N])
{
    return {v, (int)N};
}

}  // namespace

VariantList variants_f64(int Q)
{
    switch (Q) {
    case 1: return list(kF64Q1);
    case 4: return list(kF64Q4);
    case 8: return list(kF64Q8);
    case 27: return list(kF64Q27);
    case 64: return list(kF64Q64);
    default: return {};
    }
}

}  // namespace bs
