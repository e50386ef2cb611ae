// The batched stage kernel under its lowest register budget (BATCH_LO: at most 64 registers a thread);
// its own translation unit so that the budgets compile in parallel.
#include "gdg_batch_kernel.cuh"

namespace gdg_batch_dev {

extern const BatchOps batch_ops_lo = batch_ops_of<BATCH_LO>();

}  // namespace gdg_batch_dev
