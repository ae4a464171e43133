// float32 instantiations of the fused filter kernels (kernels in filter_impl.cuh).
#include "filter_impl.cuh"

namespace mm {

void launch_filter_fft_f32(const FilterArgs& a, bool from_tod, cudaStream_t s) {
    if (a.half) {
        if (from_tod) launch_half_t<float, true>(a, s);
        else launch_half_t<float, false>(a, s);
    } else {
        if (from_tod) launch_fft_t<float, true>(a, s);
        else launch_fft_t<float, false>(a, s);
    }
}
void launch_filter_direct_f32(const FilterArgs& a, bool from_tod, cudaStream_t s) {
    if (from_tod) launch_direct_t<float, true>(a, s);
    else launch_direct_t<float, false>(a, s);
}

}  // namespace mm
