// N-body with merging collisions (Fig. 6b/6d): placeholder dispatch until
// the application is built.
#include "dsr_internal.cuh"

int dsr__nbody_method(dsr_heap*, int, int, const void*, size_t, cudaStream_t, bool) { return DSR_E_INVALID; }
