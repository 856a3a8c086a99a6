// Split-precision exchange (filled in below the FP64 path).
#include "common.cuh"

namespace dfhf {

void exchange_split(df_handle* h, int nocc, int slices, double* dK) {
    (void)h; (void)nocc; (void)slices; (void)dK;
    throw Error{DF_E_ARG, "split-precision exchange is not available in this build"};
}

void free_split(df_handle* h) { (void)h; }

}  // namespace dfhf
