// raster_c32.cu -- compositing kernels for 32 semantic channels (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace sg {
template sg_status launch_raster_c<32>(RasterArgs &, bool, cudaStream_t);
}  // namespace sg
