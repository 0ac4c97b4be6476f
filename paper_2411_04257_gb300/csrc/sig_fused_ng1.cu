#define LSHB_NG 1
#include "sig_fused_inst.cuh"
