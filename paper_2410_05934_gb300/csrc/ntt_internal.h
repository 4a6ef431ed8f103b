// Internal plan representation shared by the host plan builder, the C ABI,
// the kernel launchers and the host emulation.  Not part of the public ABI.
#pragma once
#include <stdint.h>
#include <mutex>
#include <string>
#include <vector>

#include "ntt_gb300.h"
#include "ntt_tile.cuh"
#include "ntt32.cuh"

namespace nttgb {

// Host-side number theory of the plan (Sec. II-D: q prime, q = 1 mod 2N,
// psi a primitive 2N-th root of unity).  Independent of any test oracle.
bool is_prime_u64(uint64_t n);
uint64_t pow_mod(uint64_t a, uint64_t e, uint64_t q);
uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t q);
int jacobi(uint64_t a, uint64_t n);
uint64_t root_2n(uint64_t q, uint32_t log2n);
uint64_t shoup_of(uint64_t w, uint64_t q);

struct PlanHost {
    uint32_t log2n = 0, n_moduli = 0, batch = 0, flags = 0;
    uint32_t mc = 0;                   // modulus class (see ntt_tile.cuh)
    uint64_t rows = 0;
    std::vector<uint64_t> moduli, psi;
    std::vector<TwPair> fwd, inv;      // [n_moduli][N]
    std::vector<LimbConst> consts;     // [n_moduli]
    std::vector<LimbConst> consts_mont;   // the same with the last-stage scale times 2^64
    std::vector<TwPair> otf_fwd, otf_inv;   // NTT_FLAG_OTF_TWIDDLES: [n_moduli][otf_entries(log2n)]
    std::vector<Tw32> fwd32, inv32;    // NTT_FLAG_WORD32 plans: 32-bit tables
    std::vector<LimbConst32> consts32;
};

// Validates the arguments and fills the host tables.  Returns NTT_OK or an
// NTT_ERR_* code.
int build_plan_host(PlanHost& h, uint32_t log2n, const uint64_t* moduli, uint32_t n_moduli,
                    uint32_t batch, uint32_t flags);

// Constant block of an RNS basis conversion Q -> P (layout in rns.cuh) and
// the number of 128-bit terms one accumulator may hold.
int bconv_constants(const uint64_t* q_from, uint32_t L, const uint64_t* p_to, uint32_t K,
                    std::vector<uint64_t>& w, uint32_t& chunk);

// ---- schedules ----
struct ScheduleInfo {
    uint32_t log2n;
    uint32_t kernels;      // launches per transform
    const char* name;
};
// candidate schedules of one N, in table order; default_schedule() picks one
int schedule_count(uint32_t log2n);
const ScheduleInfo* schedule_info(uint32_t log2n, uint32_t id);
uint32_t default_schedule(uint32_t log2n, uint64_t rows);

}  // namespace nttgb

struct ntt_plan_s {
    nttgb::PlanHost h;
    int device = -1;
    nttgb::TwPair* d_fwd = nullptr;
    nttgb::TwPair* d_inv = nullptr;
    nttgb::LimbConst* d_consts = nullptr;
    nttgb::LimbConst* d_consts_mont = nullptr;
    int* d_status = nullptr;
    nttgb::Tw32* d_fwd32 = nullptr;
    nttgb::Tw32* d_inv32 = nullptr;
    nttgb::LimbConst32* d_consts32 = nullptr;
    nttgb::TwPair* d_otf_fwd = nullptr;
    nttgb::TwPair* d_otf_inv = nullptr;
    uint32_t schedule = 0;
    uint32_t last_launches = 0;
    // the two-stream row split of two-kernel schedules (device plans of
    // 64-bit words): a non-blocking side stream and its fork / join events
    // (cudaStream_t / cudaEvent_t), and the lock that keeps one call's
    // record / wait pairs together when several host threads share the plan
    void* side = nullptr;
    void* ev_fork = nullptr;
    void* ev_join = nullptr;
    std::mutex split_mu;
};
