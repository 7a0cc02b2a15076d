// Warm-start network kernels (filled in by the warm-start path).
#include "fcm_runtime.h"

void fcm_release_mlp(fcm_ctx* h) { (void)h; }
