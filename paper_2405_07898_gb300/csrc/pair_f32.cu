// pair_f32.cu -- density and force passes with float pair arithmetic.
#include "pair_kernels.cuh"

namespace eammd {
template int launch_density<float>(const Bufs<float> &, const Geom &, const Launch &, bool);
template int launch_force<float>(const Bufs<float> &, const Geom &, const Launch &, int, bool);
}  // namespace eammd
