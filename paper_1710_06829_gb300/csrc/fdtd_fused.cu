// placeholder, replaced by the fused kernel
#include "fdtd_internal.cuh"
namespace fdtd {
template <typename T>
bool fused_supported(const Geom&) { return false; }
template <typename T>
void launch_step_fused(const Geom&, const Mult<T>&, FieldSet<T>, FieldSet<T>, const T*, const T*,
                       const T*, const T*, T* [3], cudaStream_t) {}
template bool fused_supported<float>(const Geom&);
template bool fused_supported<double>(const Geom&);
template void launch_step_fused<float>(const Geom&, const Mult<float>&, FieldSet<float>, FieldSet<float>, const float*, const float*, const float*, const float*, float* [3], cudaStream_t);
template void launch_step_fused<double>(const Geom&, const Mult<double>&, FieldSet<double>, FieldSet<double>, const double*, const double*, const double*, const double*, double* [3], cudaStream_t);
}
