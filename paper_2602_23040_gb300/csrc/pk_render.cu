// Convenience entry points that chain the calls of one iteration: the
// forward a1 -> a2 -> a3 -> a4 and the backward a5 -> a6, all enqueued on
// one stream (no extra work, no synchronisation).
#include "pk_common.cuh"

extern "C" pk_status pk_render_fwd(const pk_plan *p, const void *atlas, const uint32_t *occ, const uint32_t *dyn,
                                   float *soa, uint32_t *texel, uint8_t *dynflag, float *records,
                                   uint32_t *sorted_vals, uint64_t *tile_ranges, float *image, float *T_final,
                                   uint32_t *n_contrib, void *ws, pk_stream_t stream) {
  pk_status e = pk_atlas_gather(p, atlas, occ, dyn, soa, texel, dynflag, ws, stream);
  if (e == PK_OK) e = pk_project_and_sh(p, soa, records, ws, stream);
  if (e == PK_OK) e = pk_bin_and_sort(p, records, sorted_vals, tile_ranges, ws, stream);
  if (e == PK_OK) e = pk_rasterize_fwd(p, records, sorted_vals, tile_ranges, image, T_final, n_contrib, ws, stream);
  return e;
}

extern "C" pk_status pk_render_bwd(const pk_plan *p, const float *soa, const uint8_t *dynflag, const uint32_t *texel,
                                   const float *records, const uint32_t *sorted_vals, const uint64_t *tile_ranges,
                                   const float *T_final, const uint32_t *n_contrib, const float *dL_dimage,
                                   float *grad2d, float *grad_atlas, int32_t accumulate, void *ws,
                                   pk_stream_t stream) {
  pk_status e = pk_rasterize_bwd(p, records, sorted_vals, tile_ranges, T_final, n_contrib, dL_dimage, grad2d, ws,
                                 stream);
  if (e == PK_OK) e = pk_atlas_scatter_grad(p, soa, grad2d, dynflag, texel, grad_atlas, accumulate, ws, stream);
  return e;
}
