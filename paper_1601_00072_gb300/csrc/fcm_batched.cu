// Batched FCM over many independent slices (filled in by the batched path).
#include "fcm_runtime.h"

void fcm_release_batched(fcm_ctx* h) { (void)h; }
