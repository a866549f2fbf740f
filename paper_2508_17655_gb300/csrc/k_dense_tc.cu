// k_dense_tc.cu -- tcgen05 (5th-generation tensor core) path: placeholder
// until the fused kernel lands.
#include "gsb_internal.cuh"

namespace gsb {
bool tc_available() { return false; }
gsb_status tc_setup(gsb_run_state*) { return set_error(GSB_EUNSUPPORTED, "tcgen05 path not built"); }
gsb_status tc_steps(gsb_run_state*, int, int) { return set_error(GSB_EUNSUPPORTED, "tcgen05 path not built"); }
gsb_status tc_energy(gsb_run_state*) { return set_error(GSB_EUNSUPPORTED, "tcgen05 path not built"); }
void tc_free(gsb_run_state*) {}
}  // namespace gsb
