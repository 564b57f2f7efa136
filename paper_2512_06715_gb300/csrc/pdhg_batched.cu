// Batched node LPs sharing K (branch-and-bound relaxations).
#include "internal.cuh"

extern "C" int pdhg_solve_batched(void* ws, int32_t B, const double* l_b, const double* u_b,
                                  double* x_out, double* y_out, pdhg_result* res_b, void* stream) {
  (void)ws; (void)B; (void)l_b; (void)u_b; (void)x_out; (void)y_out; (void)res_b; (void)stream;
  return PDHG_ERR_UNSUPPORTED;
}
