// Register-phased program of a shared-memory kernel (host compiler output,
// device interpreter input).  See shm_program.cpp for the scheme.
#pragma once

#include <cstdint>
#include <vector>

namespace qs {

constexpr int kRegBits = 5;          // register qubits per thread: 32 amplitudes
constexpr int kRegAmps = 1 << kRegBits;
constexpr int kMaxThreadBits = 9;    // 2^14 tile / 32 per thread = 512 threads
constexpr int kMinPhasedM = 10;      // smaller tiles use the generic kernel

// opcodes of the program stream (uint32 words; word 0 = op | a<<8 | b<<16 | c<<24)
enum : uint32_t {
  PK_END = 0,
  PK_G1 = 1,    // a = slot, b = control ref; 8 floats (2x2 complex)
  PK_XG = 2,    // a = slot, b = control ref; swap the pair (X gate)
  PK_D1 = 3,    // a = slot, b = known ref (or none), c = unit mask; 8 floats d[4]
  PK_D2 = 4,    // a = slot0 < b = slot1, c = unit mask; 8 floats d[4]
  PK_D0 = 5,    // a = known ref0, b = known ref1 (or none), c = unit mask; 8 floats
  PK_SWAPR = 6, // a = slot0 < b = slot1
  PK_XX = 7,    // a = slot0 < b = slot1; 2 floats (cos t/2, sin t/2)
  PK_XCHG = 8,  // a = thread bits; 5 words er[], then nt words (tloc | tswz << 16)
};

// qubit references inside an op
constexpr uint32_t REF_NONE = 0xFF;
constexpr uint32_t REF_LOCAL = 0x40;   // | local bit (a thread bit of the phase)
constexpr uint32_t REF_GLOBAL = 0x80;  // | physical bit (a batch bit)

// Shared-memory index swizzle: XOR-fold of bits 4.. into bits 0..3.  Linear
// over GF(2), so swz(a ^ b) = swz(a) ^ swz(b).
inline uint32_t swz(uint32_t x) {
  uint32_t y = x >> 4;
  uint32_t f = y ^ (y >> 4) ^ (y >> 8) ^ (y >> 12);
  return x ^ (f & 15u);
}

struct PhaseMap {
  int R[kRegBits];           // slot i -> local bit
  int T[kMaxThreadBits];     // thread bit k -> local bit
  int nt = 0;
};

struct ShmProgramV2 {
  bool ok = false;           // false: use the generic kernel
  int m = 0;
  std::vector<uint32_t> prog;
  PhaseMap load, store;
  uint64_t ld_preg[kRegBits], ld_pthr[kMaxThreadBits];
  uint64_t st_preg[kRegBits], st_pthr[kMaxThreadBits];
  uint32_t ld_er[kRegBits], ld_tloc[kMaxThreadBits], ld_tswz[kMaxThreadBits];
  int num_phases = 0;        // exchanges + 1
  int num_ops = 0;
};

}  // namespace qs
