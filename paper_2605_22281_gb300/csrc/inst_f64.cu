// FP64 values, FP64 vectors.
#include "inst_common.cuh"
namespace sfl { template struct Ops<double, double>; }
