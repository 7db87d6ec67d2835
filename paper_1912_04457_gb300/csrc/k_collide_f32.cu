// FP32 collision path: the integrand in single precision with FMA
// contraction, uniforms with 23-bit resolution; deposits stay int64 fixed
// point, so number conservation is still exact.
#include "collide.cuh"

namespace bz {

cudaError_t launch_collide_f32(const CollideArgs<float>& a, int grid, cudaStream_t s)
{
    k_collide<float><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bz
