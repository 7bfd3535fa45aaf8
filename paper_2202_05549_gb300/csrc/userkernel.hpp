// Runtime compilation of user kernels (see userkernel.cpp).
#pragma once

#include <string>
#include <vector>

#include "kernels.cuh"
#include "lightning.h"

namespace lt {

struct UserParam {
    bool is_array = false;
    int dtype = LT_F32;
    int rank = 1;  // arrays: 1, 2 or 3
};

// Source of the user function plus the generated __global__ wrapper.
std::string user_wrapper_source(const std::string &user, const std::string &name, const std::vector<UserParam> &params);

// NVRTC compilation for sm_103a: LT_OK (cubin filled), LT_ERR_COMPILE (log
// holds the compiler messages) or LT_ERR_UNSUPPORTED (no NVRTC).
lt_status compile_user_kernel(const std::string &src, std::vector<char> *cubin, std::string *log);

namespace k {
// One CUDA block per virtual block of every superblock.
uint32_t prepare_user(ExecTask *t, int n, ExecParams &p);
}  // namespace k

}  // namespace lt
