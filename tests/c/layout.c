/* Prints the layout of the option and result structs of include/pc.h, one
 * "struct field offset" line per field and a "struct sizeof size" line per
 * struct, so that a test can compare them with the Python binding's ctypes
 * structures. */
#include <stddef.h>
#include <stdio.h>

#include "pc.h"

#define F(s, f) printf(#s " " #f " %zu\n", offsetof(s, f))
#define Z(s) printf(#s " sizeof %zu\n", sizeof(s))

int main(void) {
  F(pc_options, precision); F(pc_options, exec); F(pc_options, keep_tape); F(pc_options, strict);
  F(pc_options, init_vcap); F(pc_options, init_ecap); F(pc_options, mem_budget_bytes);
  F(pc_options, filter_kappa); F(pc_options, polish); F(pc_options, polish_tol); F(pc_options, timers);
  F(pc_options, gemm); F(pc_options, pairing); F(pc_options, canonical); F(pc_options, prune);
  F(pc_options, debug_barrier_timeout); F(pc_options, filter_kappa_audit);
  Z(pc_options);
  F(pc_server_options, max_slots); F(pc_server_options, precision); F(pc_server_options, exec);
  F(pc_server_options, polish); F(pc_server_options, keep_outputs); F(pc_server_options, mem_budget_bytes);
  F(pc_server_options, request_max_bytes);
  Z(pc_server_options);
  F(pc_result, status); F(pc_result, n_vertices); F(pc_result, n_edges); F(pc_result, arrival_s);
  F(pc_result, start_s); F(pc_result, finish_s); F(pc_result, est_bytes); F(pc_result, slot);
  F(pc_result, held_bytes);
  Z(pc_result);
  return 0;
}
