// raster.cu -- dispatch of the compositing kernels (raster_impl.cuh) over the semantic
// width C; each C is instantiated in its own translation unit (raster_c*.cu) so that
// they compile in parallel.
#include "raster.cuh"

namespace sg {

template <int C>
sg_status launch_raster_c(RasterArgs &a, bool backward, cudaStream_t st);

extern template sg_status launch_raster_c<4>(RasterArgs &, bool, cudaStream_t);
extern template sg_status launch_raster_c<8>(RasterArgs &, bool, cudaStream_t);
extern template sg_status launch_raster_c<16>(RasterArgs &, bool, cudaStream_t);
extern template sg_status launch_raster_c<32>(RasterArgs &, bool, cudaStream_t);
extern template sg_status launch_raster_c<40>(RasterArgs &, bool, cudaStream_t);

sg_status launch_raster(RasterArgs &a, int C, bool backward, cudaStream_t st) {
    switch (C) {
        case 4: return launch_raster_c<4>(a, backward, st);
        case 8: return launch_raster_c<8>(a, backward, st);
        case 16: return launch_raster_c<16>(a, backward, st);
        case 32: return launch_raster_c<32>(a, backward, st);
        case 40: return launch_raster_c<40>(a, backward, st);
        default:
            set_error("unsupported semantic width C=%d (supported: 4, 8, 16, 32, 40)", C);
            return SG_ERR_INVALID_ARG;
    }
}

bool raster_supports(int C) { return C == 4 || C == 8 || C == 16 || C == 32 || C == 40; }

}  // namespace sg
