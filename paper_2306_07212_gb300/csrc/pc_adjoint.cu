// Adjoint of the vertex coordinates w.r.t. the network parameters.
#include "pc.h"
#include "pc_ctx.h"

extern "C" pc_status pc_backward(pc_ctx* c, const double* grad_x, double* grad_params, void* stream) {
  if (!c || !grad_x || !grad_params) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (!c->opt.keep_tape) return c->fail(PC_ERR_NO_TAPE, "extraction ran without keep_tape");
  (void)stream;
  return c->fail(PC_ERR_INVALID, "adjoint not available in this build");
}
