// Entry points whose implementation is not in this build yet.
#include "runtime.h"

using namespace sdfg;

extern "C" int sdfg_jacobi2d_solve(sdfg_desc *, int, const sdfg_config *, void *) {
    return set_error(SDFG_ERR_UNSUPPORTED, "sdfg_jacobi2d_solve is not built yet");
}
extern "C" int sdfg_jacobi2d_batch(sdfg_desc *, int, int, void *) {
    return set_error(SDFG_ERR_UNSUPPORTED, "sdfg_jacobi2d_batch is not built yet");
}
extern "C" int sdfg_batch_plan_create(sdfg_batch_plan **, const sdfg_desc *, int, int, const sdfg_config *, void *) {
    return set_error(SDFG_ERR_UNSUPPORTED, "batch plans are not built yet");
}
extern "C" int sdfg_batch_plan_run(sdfg_batch_plan *, void *) { return SDFG_ERR_UNSUPPORTED; }
extern "C" int sdfg_batch_plan_results(sdfg_batch_plan *, sdfg_desc *, int) { return SDFG_ERR_UNSUPPORTED; }
extern "C" int sdfg_batch_plan_destroy(sdfg_batch_plan *) { return SDFG_ERR_UNSUPPORTED; }
extern "C" int sdfg_server_create(sdfg_server **, size_t, int, int, int, int) { return SDFG_ERR_UNSUPPORTED; }
extern "C" int sdfg_server_submit(sdfg_server *, const sdfg_desc *, uint64_t *) { return SDFG_ERR_UNSUPPORTED; }
extern "C" int sdfg_server_poll(sdfg_server *, uint64_t, sdfg_desc *) { return SDFG_ERR_UNSUPPORTED; }
extern "C" int sdfg_server_drain(sdfg_server *, int) { return SDFG_ERR_UNSUPPORTED; }
extern "C" int sdfg_server_destroy(sdfg_server *) { return SDFG_ERR_UNSUPPORTED; }
