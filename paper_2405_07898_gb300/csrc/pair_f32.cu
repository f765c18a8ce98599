// pair_f32.cu -- density and force passes with float pair arithmetic.
#include "pair_kernels.cuh"

#include <algorithm>

namespace eammd {
template int launch_density<float>(const Bufs<float> &, const Geom &, const Launch &, bool);
template int launch_force<float>(const Bufs<float> &, const Geom &, const Launch &, int, bool);
template cudaError_t allow_shared_staging<float>(int);

int table_grid(const Launch &L, bool force, int tpa, int block)
{
    const int per_sm = table_blocks_per_sm(L, force, tpa, block);
    int dev = 0, nsm = 0;
    if (per_sm <= 0 || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    const int width = block / tpa;
    const int ntiles = (L.n + width - 1) / width;
    return std::max(1, std::min(ntiles, per_sm * nsm));
}

}  // namespace eammd
