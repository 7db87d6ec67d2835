// FP64 collision path.  Compiled with -fmad=false: each operation of the
// formula is one IEEE-rounded step in the written order (division and sqrt
// are correctly rounded in FP64), so the int64 deposits are bit-identical
// to the FP64 CPU oracle's.
#include "collide.cuh"

namespace bz {

cudaError_t check_read_collide_f64(unsigned long long out[2], bool reset)
{
#if BZ_CHECK
    cudaError_t e = cudaMemcpyFromSymbol(out, g_bz_check, 2 * sizeof(unsigned long long));
    const unsigned long long zero[2] = {0ull, 0ull};
    if (e == cudaSuccess && reset) e = cudaMemcpyToSymbol(g_bz_check, zero, sizeof(zero));
    return e;
#else
    out[0] = out[1] = 0ull;
    (void)reset;
    return cudaErrorNotSupported;
#endif
}

cudaError_t launch_collide_f64(const CollideArgs<double>& a, int grid, cudaStream_t s)
{
    k_collide<double><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bz
