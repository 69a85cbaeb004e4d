// bs_vel_exact.cu -- instances of the velocity kernel whose near pairs take the exact integral of Eq. 1
// over the tet (near_rule = BS_NEAR_EXACT), both precisions.
#include "bs_velocity_kernel.cuh"

namespace bs {
namespace {

#define BS_V(T, Q, P, TILE, S, MINB, INL) \
    { {P, TILE, S, MINB, INL, 1, false, 1}, &launch_t<T, Q, P, 128, TILE, S, MINB, INL, true, 1, false, 1> }

const VariantEntry kF32Q1[] = {BS_V(float, 1, 2, 32, 4, 4, true)};
const VariantEntry kF32Q4[] = {BS_V(float, 4, 3, 32, 2, 4, true), BS_V(float, 4, 1, 32, 4, 5, false)};
const VariantEntry kF32Q8[] = {BS_V(float, 8, 2, 16, 4, 4, true)};
const VariantEntry kF32Q27[] = {BS_V(float, 27, 1, 16, 4, 4, false)};
const VariantEntry kF32Q64[] = {BS_V(float, 64, 1, 8, 4, 4, false)};
const VariantEntry kF64Q1[] = {BS_V(double, 1, 2, 32, 4, 4, true)};
const VariantEntry kF64Q4[] = {BS_V(double, 4, 1, 32, 2, 4, true), BS_V(double, 4, 2, 32, 2, 3, true)};
const VariantEntry kF64Q8[] = {BS_V(double, 8, 2, 16, 4, 4, true)};
const VariantEntry kF64Q27[] = {BS_V(double, 27, 1, 16, 4, 4, false)};
const VariantEntry kF64Q64[] = {BS_V(double, 64, 1, 8, 4, 4, false)};
#undef BS_V

template <size_t N>
VariantList list(const VariantEntry (&v)[N])
{
    return {v, (int)N};
}

}  // namespace

VariantList variants_exact(int precision, int Q)
{
    const bool f32 = precision == BS_FP32;
    switch (Q) {
    case 1: return f32 ? list(kF32Q1) : list(kF64Q1);
    case 4: return f32 ? list(kF32Q4) : list(kF64Q4);
    case 8: return f32 ? list(kF32Q8) : list(kF64Q8);
    case 27: return f32 ? list(kF32Q27) : list(kF64Q27);
    case 64: return f32 ? list(kF32Q64) : list(kF64Q64);
    default: return {};
    }
}

}  // namespace bs
