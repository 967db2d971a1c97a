// msz_edits_async.h -- the edit-list encoder queued behind a correction on a
// stream, with the edit count read on the device (used by the pipelined
// host-buffer entry points).  Internal: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "msz.h"
#include "msz_workspace.h"

namespace msz {

// Device workspace of encode_async for up to count_cap edits; its first 16
// bytes hold {uint32 error, uint32 pad, uint64 total_words} once the encode
// has run.
size_t encode_async_workspace(uint64_t count_cap);

// Length of the stream of `count` edits whose payload has total_words words.
uint64_t encoded_length(uint64_t count, uint64_t total_words);

// Encodes the edit list d_idx[0 .. min(*d_count, count_cap)) of g = d_g
// against d_fhat into d_stream (capacity bytes) on stream s.  A nonzero error
// in the workspace afterwards means nothing was written (bit 1: bad indices,
// bit 2: the stream would exceed capacity).
msz_status encode_async(const float *d_fhat, const float *d_g, uint32_t n, const uint32_t *d_idx,
                        const unsigned long long *d_count, uint64_t count_cap, uint8_t *d_stream, size_t capacity,
                        void *d_ws, const DeviceInfo &dev, cudaStream_t s);

// Copies the stream that encode_async wrote (d_stream, its state in d_ws)
// into host memory that the device can address (h_dst: its device pointer,
// capacity bytes), on stream s: the length is known on the device only, so
// a kernel writes it there, and no copy engine is queued behind the
// correction (an upload queued behind a download that waits for a kernel
// would wait with it).  Nothing is written when the encode reported an error
// or the stream exceeds the capacity (the host sees both in the state).
msz_status stream_out_async(const uint8_t *d_stream, const void *d_ws, const unsigned long long *d_count,
                            uint64_t count_cap, uint8_t *h_dst, size_t capacity, cudaStream_t s);

}  // namespace msz
