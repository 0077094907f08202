// Grid-side kernels of the PIC step: metric tables at the Yee points.
#include "fpic_internal.h"

namespace fpic {

int build_metric_tables(fpic_ctx* c)
{
    (void)c;
    return 0;
}

}  // namespace fpic
