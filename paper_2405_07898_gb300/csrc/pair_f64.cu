// pair_f64.cu -- density and force passes with double pair arithmetic.
#include "pair_kernels.cuh"

namespace eammd {
template int launch_density<double>(const Bufs<double> &, const Geom &, const Launch &, bool);
template int launch_force<double>(const Bufs<double> &, const Geom &, const Launch &, int, bool);
}  // namespace eammd
