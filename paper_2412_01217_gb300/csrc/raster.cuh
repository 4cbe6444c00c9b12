// raster.cuh -- launch arguments of the tile compositing kernels (raster.cu), shared with
// the C-ABI layer.
#pragma once

#include "sg_common.cuh"

namespace sg {

struct RasterArgs {
    const float4 *geo;
    const float2 *ext;
    const uint32_t *record;
    const int2 *ranges;
    const int *order;  // work order of the tiles (null: id order)
    const float *rgb;  // colour: N x 3 per Gaussian, or R x 3 per record when col_rec
    int col_rec;       // 1: colour (and its gradient) indexed by record, else by Gaussian
    const float *sem;  // semantic feature: N x C per Gaussian, or R x C per record when sem_rec
    int sem_rec;       // 1: semantic feature (and its gradient) indexed by record
    const sg_view *views;
    int n_views, n_tiles, N;
    float alpha_max, alpha_min, T_min;
    float bg0, bg1, bg2;
    int tile_w, tile_h, batch;
    int *work_counter;
    int persistent;
    int ppt;  // pixels per thread (1, 2 or 4)
    int half;             // records carry half masks in bits 30-31: the adjoint of 8 x 8
                          // tiles at one pixel per thread runs one warp per half tile
    int half_fwd;         // ... and so does the forward (sg_config.half_tile_fwd)
    int half_pairs;       // half-tile adjoint: a work item is a whole tile, both halves in turn
    uint32_t rec_mask;    // bits of a list word that hold the record id
    // forward outputs / backward inputs
    float *img_rgb, *img_depth, *img_sem;
    float *T_final;
    int *last, *n_contrib;
    // backward
    const float *dL_rgb, *dL_depth, *dL_sem;
    float *g2d, *g_sem;
    float *g_col;    // colour gradient: col_stride floats per Gaussian (or record when col_rec)
    int col_stride;
    int sem_v2;  // g_sem is 8-byte aligned (pairs of semantic gradients in one vector reduction)
};

inline void fill_raster_args(RasterArgs &a, const sg_gaussians *g, const sg_projected *proj,
                             const sg_tile_lists *lists, const sg_view *views, int n_views,
                             int n_tiles, const sg_config *cfg, int *work_counter) {
    a.geo = reinterpret_cast<const float4 *>(proj->geo);
    a.ext = reinterpret_cast<const float2 *>(proj->ext);
    a.record = lists->record;
    a.ranges = reinterpret_cast<const int2 *>(lists->ranges);
    a.order = lists->order;
    a.col_rec = g->sh_degree > 0 && g->sh;
    a.rgb = a.col_rec ? proj->rgb : g->rgb;
    a.sem_rec = g->sh_degree > 0 && g->sem_sh;
    a.sem = a.sem_rec ? proj->sem : g->sem;
    a.views = views;
    a.n_views = n_views;
    a.n_tiles = n_tiles;
    a.N = g->N;
    a.alpha_max = cfg->alpha_max;
    a.alpha_min = cfg->alpha_min;
    a.T_min = cfg->T_min;
    a.bg0 = cfg->bg[0];
    a.bg1 = cfg->bg[1];
    a.bg2 = cfg->bg[2];
    a.tile_w = cfg->tile_w;
    a.tile_h = cfg->tile_h;
    a.batch = cfg->batch;
    a.work_counter = work_counter;
    a.persistent = cfg->persistent;
    a.ppt = cfg->pixels_per_thread;
    a.half = lists->half_masks != 0;
    a.half_fwd = cfg->half_tile_fwd != 0;
    a.rec_mask = a.half ? 0x3fffffffu : 0xffffffffu;
}

sg_status launch_raster(RasterArgs &a, int C, bool backward, cudaStream_t st);
bool raster_supports(int C);

}  // namespace sg
