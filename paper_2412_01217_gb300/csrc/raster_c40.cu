// raster_c40.cu -- compositing kernels for 40 semantic channels (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace sg {
template sg_status launch_raster_c<40>(RasterArgs &, bool, cudaStream_t);
}  // namespace sg
