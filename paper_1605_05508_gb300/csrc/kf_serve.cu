// kf_serve.cu -- serving loop (continuous batching); placeholder teardown.
#include "kf_internal.h"
void kf_serve_shutdown_internal(kf_ctx* ctx) { (void)ctx; }
