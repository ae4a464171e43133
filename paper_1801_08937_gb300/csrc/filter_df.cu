// Double-float instantiations of the fused filter kernels (kernels in filter_impl.cuh).
#include "filter_impl.cuh"

namespace mm {

void launch_filter_fft_df(const FilterArgs& a, bool from_tod, cudaStream_t s) {
    if (a.half) {
        if (from_tod) launch_half_t<df, true>(a, s);
        else launch_half_t<df, false>(a, s);
    } else {
        if (from_tod) launch_fft_t<df, true>(a, s);
        else launch_fft_t<df, false>(a, s);
    }
}
void launch_filter_direct_df(const FilterArgs& a, bool from_tod, cudaStream_t s) {
    if (from_tod) launch_direct_t<df, true>(a, s);
    else launch_direct_t<df, false>(a, s);
}

}  // namespace mm
