// FP64 collision path.  Compiled with -fmad=false: each operation of the
// formula is one IEEE-rounded step in the written order (division and sqrt
// are correctly rounded in FP64), so the int64 deposits are bit-identical
// to the FP64 CPU oracle's.  Also hosts the FP64 re-evaluation of the terms
// the FP32 kernel queued as ill-conditioned.
#include "collide.cuh"

namespace bz {

cudaError_t launch_collide_f64(const CollideArgs<double>& a, int grid, cudaStream_t s)
{
    k_collide<double, false><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fixup(const CollideArgs<double>& a, int nseg, cudaStream_t s)
{
    k_fixup<double><<<nseg, 256, 0, s>>>(a, a.qcount, a.qitems, a.qcap);
    return cudaGetLastError();
}


}  // namespace bz
