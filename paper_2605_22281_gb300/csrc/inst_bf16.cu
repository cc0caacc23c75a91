// BF16 values, FP32 vectors.
#include "inst_common.cuh"
namespace sfl { template struct Ops<__nv_bfloat16, float>; }
