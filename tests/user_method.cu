// A method written by a user of the library against the public headers
// only (dsr.h, dsr_device.cuh): it scales field 0 of every object of a type
// and creates a new object of the same type where the value passes 100.
// tests/test_abi.py compiles it for sm_103a; it is not part of the library.
#include <cstring>
#include "dsr.h"
#include "dsr_device.cuh"
struct ScaleArgs { float scale; };
struct MScale {
    typedef ScaleArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref self) {
        float* f = dsr_field<float>(H, T, self, 0);
        *f *= a.scale;
        if (*f > 100.f) {
            const dsr_ref c = dsr_new(H, T);
            if (c != DSR_NULL) *dsr_field<float>(H, T, c, 0) = 1.f;
        }
    }
};
// A do-all over type T: the library's scan lists the live blocks, then the
// method kernel runs over the list (the run resets it).
extern "C" int user_scale(dsr_heap* heap, int T, float scale, int grid, cudaStream_t s) {
    dsr_dev_heap H;
    if (dsr_dev_heap_size() != sizeof H) return -1;
    int rc = dsr_heap_device_view(heap, &H, sizeof H);
    if (!rc) rc = dsr_doall_scan(heap, T, s);
    if (rc) return rc;
    dsr_doall_kernel<MScale><<<grid, 256, 0, s>>>(H, T, ScaleArgs{scale}, 0);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
