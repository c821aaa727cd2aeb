// Tracing of the matvec passes with CUDA events, and a count of the
// library's kernel launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace dda {

// every kernel launch of the library passes through DDA_LAUNCH_CHECK, which
// adds one here
void note_launches(int64_t n);
int64_t launch_count();

// Records a pair of events around each pass of every matvec while enabled;
// read() waits for them and sums the elapsed time per (dtype, pass).
struct PassProfiler {
    static constexpr int kPasses = 5;
    struct Rec { int dtype, pass; cudaEvent_t a, b; };
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> recs;

    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void begin(int dtype, int pass, cudaStream_t st) {
        Rec r{dtype, pass, next(), next()};
        cudaEventRecord(r.a, st);
        recs.push_back(r);
    }
    void end(cudaStream_t st) { cudaEventRecord(recs.back().b, st); }
    // counts[dtype][pass], ms[dtype][pass]; clears the records
    int read(int64_t* counts, double* ms) {
        for (int i = 0; i < 2 * kPasses; ++i) { counts[i] = 0; ms[i] = 0.0; }
        for (const Rec& r : recs) {
            if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
            float t = 0.f;
            cudaEventElapsedTime(&t, r.a, r.b);
            counts[r.dtype * kPasses + r.pass] += 1;
            ms[r.dtype * kPasses + r.pass] += t;
        }
        recs.clear();
        used = 0;
        return 0;
    }
    ~PassProfiler() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

}  // namespace dda
