// placeholder: replaced by the batched solver
#include "mst_internal.h"
namespace mst {
size_t batched_bytes(int32_t, uint64_t, uint64_t) { return 0; }
cudaError_t batched_reserve(Batched &, int32_t, uint64_t, uint64_t) { return cudaErrorNotSupported; }
void batched_release(Batched &b) { b = Batched(); }
cudaError_t batched_launch(Batched &, int, uint32_t, int32_t, const int64_t *, const int64_t *, uint64_t, uint64_t,
                           const int32_t *, const int32_t *, const void *, int32_t *, int64_t *, cudaStream_t) { return cudaErrorNotSupported; }
uint32_t batched_status_bits(Batched &, cudaStream_t, cudaError_t *err) { *err = cudaSuccess; return 0; }
mst_status server_start(mst_handle, int, int) { return MST_ERR_INTERNAL; }
mst_status server_submit(mst_handle, const Request &, uint64_t *) { return MST_ERR_INTERNAL; }
mst_status server_poll(mst_handle, uint64_t, int *, double *) { return MST_ERR_INTERNAL; }
mst_status server_drain(mst_handle) { return MST_ERR_INTERNAL; }
mst_status server_stop(mst_handle) { return MST_ERR_INTERNAL; }
}
extern "C" mst_status mst_autotune_batched(mst_handle, mst_weight_type, int32_t, const int64_t *, const int64_t *, int64_t, int64_t,
   const int32_t *, const int32_t *, const void *, int32_t *, int64_t *, const char *, void *) { return MST_ERR_INTERNAL; }
