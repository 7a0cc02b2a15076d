// Kernel table of the single-image run that recomputes U^{k-1} instead of
// storing it (fcm_recompute_inst.cu, compiled once per cluster count).
#pragma once

#include "fcm_internal.h"

namespace fcm {

struct RcTable {
    // [C][m kind][0 = from U^0, 1 = from V^0]
    RunFn run[FCM_MAX_CLUSTERS + 1][4][2];
    int smem[FCM_MAX_CLUSTERS + 1][2];
};

void register_rc_c1(RcTable&);
void register_rc_c2(RcTable&);
void register_rc_c3(RcTable&);
void register_rc_c4(RcTable&);
void register_rc_c5(RcTable&);
void register_rc_c6(RcTable&);
void register_rc_c7(RcTable&);
void register_rc_c8(RcTable&);

}  // namespace fcm
