// Proposal network for seeding the best-so-far distance (not in the paper).
#include "sofa_internal.cuh"

namespace sofa {

struct Mlp {
  int dummy;
};

void mlp_free(Mlp* m) { delete m; }

}  // namespace sofa

using namespace sofa;

extern "C" int sofa_train_proposal(sofa_handle h, const sofa_train_opts* o, sofa_stream stream) {
  (void)o;
  (void)stream;
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  return fail(SOFA_ERR_INVALID_ARG, "the proposal network is not part of this build yet");
}

extern "C" int sofa_set_seed_mode(sofa_handle h, int32_t mode) {
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  if (mode == 0) {
    h->seed_mode = 0;
    return 0;
  }
  if (mode == 1) return fail(SOFA_ERR_NOT_TRAINED, "learned seeding needs sofa_train_proposal first");
  return fail(SOFA_ERR_INVALID_ARG, "seed mode must be 0 or 1");
}
