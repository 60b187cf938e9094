// Launch profiler scope (see profile.cu).  Construct immediately before a
// kernel launch on stream st; the destructor records the end event.
#pragma once
#include <cuda_runtime.h>

class LuProfScope {
   public:
    LuProfScope(cudaStream_t st, int cls, double bytes, double flops);
    ~LuProfScope();
    LuProfScope(const LuProfScope&) = delete;
    LuProfScope& operator=(const LuProfScope&) = delete;

   private:
    cudaStream_t st_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    int cls_ = 0;
    double bytes_ = 0, flops_ = 0;
    bool active_ = false;
};
