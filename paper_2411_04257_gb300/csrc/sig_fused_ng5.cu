#define LSHB_NG 5
#include "sig_fused_inst.cuh"
