// Host-side utilities shared by the planner, executor, driver and C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/bbtn.h"

namespace bbtn {

// thread-local message of the last failure (bbtn_last_error)
void set_error(const std::string &msg);
const char *get_error();

// An exception carrying a BBTN_E* code; converted to a return code at the C ABI.
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string &msg) { throw Error{code, msg}; }

#define BBTN_CUDA(call)                                                                     \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            ::bbtn::fail(e_ == cudaErrorMemoryAllocation ? BBTN_ENOMEM : BBTN_ECUDA,        \
                         std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

inline double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ primes / CRT
// Primes p_t = 2^61 - c_t (c_t ascending) found by deterministic Miller-Rabin.
// Index kCheckPrime is reserved for the overflow guard.
constexpr int kCheckPrime = BBTN_MAX_PRIMES;
const std::vector<uint64_t> &prime_table();     // BBTN_MAX_PRIMES + 1 entries
// Primes q = 2^30 - d (d ascending, d < 2^10) for count planes that hold two residues:
// plane t of the pair form takes q[2t] (low half) and q[2t + 1] (high half), and the
// check plane q[2 kCheckPrime], q[2 kCheckPrime + 1].
const std::vector<uint64_t> &pair_prime_table();   // 2 (BBTN_MAX_PRIMES + 1) entries
bool is_prime_u64(uint64_t n);
// Checks np plane moduli (all primes 2^61 - c, or all pairs q1 << 32 | q0 of primes
// 2^30 - d) and writes each plane's constant word for the kernels; fails on others.
void plane_moduli(int np, const uint64_t *primes, uint32_t *c);

// Garner recombination of residues r[t] mod p[t] into a decimal string.
std::string crt_decimal(const std::vector<uint64_t> &r, const std::vector<uint64_t> &p);
// the recombined integer reduced mod q
uint64_t crt_mod(const std::vector<uint64_t> &r, const std::vector<uint64_t> &p, uint64_t q);

uint64_t mulmod_host(uint64_t a, uint64_t b, uint64_t p);
uint64_t powmod_host(uint64_t a, uint64_t e, uint64_t p);

}  // namespace bbtn
