// FP32 values, FP32 vectors.
#include "inst_common.cuh"
namespace sfl { template struct Ops<float, float>; }
