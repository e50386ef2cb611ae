// The batched stage kernel under its middle register budget (BATCH_MID: at most 128 registers a thread);
// its own translation unit so that the budgets compile in parallel.
#include "gdg_batch_kernel.cuh"

namespace gdg_batch_dev {

extern const BatchOps batch_ops_mid = batch_ops_of<BATCH_MID>();

}  // namespace gdg_batch_dev
