// raster_c4.cu -- compositing kernels for 4 semantic channels (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace sg {
template sg_status launch_raster_c<4>(RasterArgs &, bool, cudaStream_t);
}  // namespace sg
