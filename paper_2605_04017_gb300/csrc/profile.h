// Kernel timing hooks (CUDA events on the launch stream); see profile.cpp.
#pragma once

#include <cuda_runtime.h>

#include "lt_internal.h"

namespace lt {

bool prof_enabled();

// Brackets the launches made during its lifetime with two events on `st`
// when profiling is on; a no-op otherwise.
class ProfScope {
public:
    ProfScope(const char* name, cudaStream_t st);
    ~ProfScope();
    // device counter for the kernel's work units while profiling, else nullptr
    unsigned long long* work() const { return work_; }
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

private:
    const char* name_;
    cudaStream_t st_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    bool active_ = false;
    unsigned long long* work_ = nullptr;
    int slot_ = -1;
};

}  // namespace lt
