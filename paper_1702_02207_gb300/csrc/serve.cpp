// serve.cpp -- continuous-batching request loop (cho_submit / cho_poll).
#include "../../include/cho.h"
#include "ctx.h"

namespace cho {
void serve_stop(cho_ctx*) {}
}  // namespace cho

using namespace cho;

extern "C" cho_status cho_submit(cho_ctx*, const cho_request*, uint64_t*)
{
    return fail(CHO_EINVAL, "cho_submit: serving is not available in this build");
}
extern "C" cho_status cho_poll(cho_ctx*, uint64_t, cho_result*)
{
    return fail(CHO_ENOTFOUND, "cho_poll: serving is not available in this build");
}
extern "C" cho_status cho_cancel(cho_ctx*, uint64_t)
{
    return fail(CHO_ENOTFOUND, "cho_cancel: serving is not available in this build");
}
extern "C" cho_status cho_serve_stats(cho_ctx*, int64_t*, int64_t*, int64_t*, int64_t*)
{
    return fail(CHO_EINVAL, "cho_serve_stats: serving is not available in this build");
}
