// raster_c8.cu -- compositing kernels for 8 semantic channels (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace sg {
template sg_status launch_raster_c<8>(RasterArgs &, bool, cudaStream_t);
}  // namespace sg
