// k_bisp.cu - the bispectrum hot path (Sec. III.B of the paper).
#include <cuda_runtime.h>

#include "fkp_internal.h"

namespace fkp {

int bisp_plan_init(Plan* P) {
  (void)P;
  return set_error(FKP_ESTATE, "bispectrum path not built in this version");
}

void bisp_plan_free(Plan* P) { (void)P; }

}  // namespace fkp

using namespace fkp;

extern "C" int fkp_bispectrum(void* plan, const fkp_catalog_t* gal, const fkp_catalog_t* ran, int contraction,
                              void* stream, fkp_power_out* pout, fkp_bisp_out* bout) {
  (void)plan; (void)gal; (void)ran; (void)contraction; (void)stream; (void)pout; (void)bout;
  return set_error(FKP_ESTATE, "bispectrum path not built in this version");
}
