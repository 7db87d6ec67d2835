// FP32 collision path: the integrand in single precision with FMA
// contraction, uniforms with 23-bit resolution; ill-conditioned terms are
// queued for FP64 re-evaluation (launch_fixup); deposits stay int64 fixed
// point, so number conservation is still exact.
#include "collide.cuh"

namespace bz {

cudaError_t launch_collide_f32(const CollideArgs<float>& a, int grid, cudaStream_t s)
{
    if (a.tau > 0.0f)
        k_collide<float, true><<<grid, 256, 0, s>>>(a);
    else
        k_collide<float, false><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bz
