// FP64 collision path.  Compiled with -fmad=false: each operation of the
// formula is one IEEE-rounded step in the written order (division and sqrt
// are correctly rounded in FP64), so the int64 deposits are bit-identical
// to the FP64 CPU oracle's.
#include "collide.cuh"

namespace bz {

cudaError_t launch_collide_f64(const CollideArgs<double>& a, int grid, cudaStream_t s)
{
    k_collide<double><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bz
