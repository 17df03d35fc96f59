// Device-side EBIC generation loop (Sec. 2.4, steps 1-9).  Filled in by the generation kernels.
#include "internal.h"

struct GenState {
  int dummy;
};

void gen_state_free(GenState *g) { delete g; }

extern "C" {

int ebic_run_generations(ebic_ctx *ctx, const ebic_params *p, int32_t n_gen,
                         ebic_run_report *rep) {
  (void)p; (void)n_gen; (void)rep;
  return ebic_fail(ctx, EBIC_ESTATE, "generation loop not available");
}
int ebic_get_toplist(ebic_ctx *ctx, int32_t capacity, int32_t *n_top, int32_t *cols,
                     int32_t *lens, uint64_t *fitness, uint64_t *keys, int32_t *rows) {
  (void)capacity; (void)n_top; (void)cols; (void)lens; (void)fitness; (void)keys; (void)rows;
  return ebic_fail(ctx, EBIC_ESTATE, "no run");
}
int ebic_get_population(ebic_ctx *ctx, int32_t capacity, int32_t *cols, int32_t *lens,
                        uint8_t *dead, uint64_t *fitness) {
  (void)capacity; (void)cols; (void)lens; (void)dead; (void)fitness;
  return ebic_fail(ctx, EBIC_ESTATE, "no run");
}
int ebic_extract_biclusters(ebic_ctx *ctx, int32_t capacity, uint32_t *rowmask, int32_t *n_out) {
  (void)capacity; (void)rowmask; (void)n_out;
  return ebic_fail(ctx, EBIC_ESTATE, "no run");
}
int64_t ebic_state_bytes(ebic_ctx *ctx) { (void)ctx; return 0; }
int ebic_save_state(ebic_ctx *ctx, void *blob, int64_t size) {
  (void)blob; (void)size;
  return ebic_fail(ctx, EBIC_ESTATE, "no run");
}
int ebic_load_state(ebic_ctx *ctx, const ebic_params *p, const void *blob, int64_t size) {
  (void)p; (void)blob; (void)size;
  return ebic_fail(ctx, EBIC_ESTATE, "no run");
}

}  // extern "C"
