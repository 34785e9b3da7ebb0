// Serving entry points (placeholder until the serving loop lands).
#include "gbd_internal.cuh"

using namespace gbd;

extern "C" {
int gbd_server_create(gbd_ctx *, const gbd_set *, gbd_server **out)
{
    if (out) *out = nullptr;
    return fail(GBD_EINVAL, "gbd_server_create: serving is not built yet");
}
int gbd_server_submit(gbd_server *, const uint8_t *, const uint64_t *, uint64_t, uint16_t *, uint64_t *)
{
    return fail(GBD_EINVAL, "gbd_server_submit: serving is not built yet");
}
int gbd_server_poll(gbd_server *, uint64_t, int *) { return fail(GBD_ENOTFOUND, "no server"); }
int gbd_server_wait(gbd_server *, uint64_t) { return fail(GBD_ENOTFOUND, "no server"); }
void gbd_server_destroy(gbd_server *) {}
}
