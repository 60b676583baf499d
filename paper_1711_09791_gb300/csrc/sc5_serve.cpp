// sc5_serve.cpp -- serving runtime (placeholder until the scheduler lands).
#include "sc5_internal.h"

namespace sc5 {
sc5_status fail(sc5_status st, const char *fmt, ...);
}
using namespace sc5;

extern "C" sc5_status serve_create(const sc5_serve_cfg *, sc5_server *) { return fail(SC5_EINVAL, "serving not built"); }
extern "C" sc5_status serve_submit(sc5_server, const sc5_image *, uint64_t *) { return fail(SC5_EINVAL, "serving not built"); }
extern "C" sc5_status serve_poll(sc5_server, uint64_t, int32_t, double *) { return fail(SC5_EINVAL, "serving not built"); }
extern "C" sc5_status serve_get_stats(sc5_server, sc5_serve_stats *) { return fail(SC5_EINVAL, "serving not built"); }
extern "C" sc5_status serve_destroy(sc5_server) { return fail(SC5_EINVAL, "serving not built"); }
