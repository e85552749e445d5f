// Temporary: batch and server entry points.
#include "lattice_capi_internal.h"
extern "C" {
int lattice_server_create(lattice_server_t **, size_t, int, int) { return LAT_ENOTSUP; }
int lattice_server_submit(lattice_server_t *, const lattice_request_t *, uint64_t *) { return LAT_ENOTSUP; }
int lattice_server_poll(lattice_server_t *, uint64_t, lattice_result_t *, int8_t *) { return LAT_ENOTSUP; }
int lattice_server_drain(lattice_server_t *, double) { return LAT_ENOTSUP; }
double lattice_server_clock(lattice_server_t *) { return 0.0; }
void lattice_server_destroy(lattice_server_t *) {}
}
