// batch.cu — batched solve of many independent grids (one persistent launch).
#include "internal.h"

extern "C" {

ps_status ps_batch_create(ps_batch** out, int, const ps_grid_desc*, ps_precision, double, int) {
  if (out) *out = nullptr;
  return PS_INVALID_ARG;
}
ps_status ps_batch_workspace_bytes(const ps_batch*, size_t* bytes) {
  if (bytes) *bytes = 0;
  return PS_INVALID_ARG;
}
ps_status ps_batch_solve(ps_batch*, double* const*, double* const*, void*, void*, ps_info*) {
  return PS_INVALID_ARG;
}
ps_status ps_batch_destroy(ps_batch*) { return PS_OK; }

}  // extern "C"
