// Adjoint of the LP solution map (implicit differentiation on the active set).
#include "internal.cuh"

extern "C" int pdhg_backward(void* ws, double g_cost, const double* g_x, double* grad_q,
                             double* grad_c, void* stream) {
  (void)ws; (void)g_cost; (void)g_x; (void)grad_q; (void)grad_c; (void)stream;
  return PDHG_ERR_UNSUPPORTED;
}
