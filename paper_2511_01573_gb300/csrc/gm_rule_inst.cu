// gm_rule_inst.cu -- instantiates the rule kernels (Genz-Malik FP64 and
// mixed, single integral and batched; tensor-product Gauss-Kronrod)
// and the adjoint kernel for one integrand family.  The build compiles this file
// once per family with -DGMQ_FAM=<code>, so the instantiations compile in
// parallel.
#include "gm_adjoint.cuh"
#include "gm_batch_mixed.cuh"
#include "gm_batch_rule64.cuh"
#include "gm_gk.cuh"
#include "gm_rule_mixed.cuh"

#ifndef GMQ_FAM
#error "compile with -DGMQ_FAM=<family code>"
#endif

namespace gmq {
GMQ_DEFINE_RULE_FAMILY(GMQ_FAM)
GMQ_DEFINE_GRAD_FAMILY(GMQ_FAM)
GMQ_DEFINE_BATCH_MIXED_FAMILY(GMQ_FAM)
GMQ_DEFINE_BATCH_RULE64_FAMILY(GMQ_FAM)
GMQ_DEFINE_GK_FAMILY(GMQ_FAM)
}  // namespace gmq
