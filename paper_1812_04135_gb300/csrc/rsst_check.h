// Caller-pointer checks of the C ABI (defined in rsst_api.cu).
#pragma once

// RSST_OK if p is memory the GPU reads as device memory (on_host = 0: a
// cudaMalloc'd or managed pointer) or host memory (on_host = 1: pageable or
// pinned); otherwise RSST_EINVAL with a message naming `where`.  A wrong
// kind of pointer would otherwise reach a kernel or a copy as an invalid
// address.
int rsst_check_buffer(const void* p, int on_host, const char* where);
