// raster_c16.cu -- compositing kernels for 16 semantic channels (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace sg {
template sg_status launch_raster_c<16>(RasterArgs &, bool, cudaStream_t);
}  // namespace sg
