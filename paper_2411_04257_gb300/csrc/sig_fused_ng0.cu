#define LSHB_NG 0
#include "sig_fused_inst.cuh"
