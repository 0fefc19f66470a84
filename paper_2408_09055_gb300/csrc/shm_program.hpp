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
constexpr int kMaxPhasedM = 14;      // 2^14 complex64 = 128 KiB tile

// opcodes of the program stream (uint32 words; word 0 = op | a<<8 | b<<16 | c<<24;
// a, b are register slots 0..4 or qubit references, c a unit-entry mask)
enum : uint32_t {
  PK_END = 0,
  PK_G1 = 1,      // a = slot; 8 floats: general 2x2 complex
  PK_G1R = 2,     // a = slot; 4 floats: real 2x2
  PK_G1X = 3,     // a = slot; 4 floats: u00 (real), u01 (imag), u10 (imag), u11 (real)
  PK_G1C = 4,     // a = slot, b = control ref; 8 floats general 2x2
  PK_XG = 5,      // a = slot: X (swap of the pair)
  PK_XGS = 6,     // a = target slot, b = control slot
  PK_XGK = 7,     // a = target slot, b = control ref known per thread
  PK_D1 = 8,      // a = slot; 4 floats: e0, e1
  PK_D1B = 9,     // a = slot; 2 floats: e1 on amplitudes with the bit set
  PK_D1K = 10,    // a = slot, b = known ref, c = unit mask; 8 floats d[bit + 2 kb]
  PK_D2 = 11,     // a = slot0 < b = slot1; 8 floats d[b0 + 2 b1]
  PK_D2P = 12,    // a = slot0 < b = slot1; 2 floats: factor on b0 = b1 = 1
  PK_D0 = 13,     // a = known ref0, b = known ref1 or none, c = unit mask; 8 floats
  PK_SWAPR = 14,  // a = slot0 < b = slot1
  PK_XX = 15,     // a = slot0 < b = slot1; 2 floats (cos t/2, sin t/2)
  PK_SCALE = 16,  // 2 floats: every amplitude times a constant
  PK_XCHG = 17,   // a = thread bits nt; 5 words er[], nt words (tloc | tswz << 16)
  PK_G2 = 18,     // a = slot0 < b = slot1; 32 floats: general 4x4, index bit(a) + 2 bit(b), row-major
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
  // global phase factored out of diagonal gates (applied once per plan)
  double phase_re = 1.0, phase_im = 0.0;
  int g1_word = -1;          // word index of the first general PK_G1's floats
  // runs of non-active bits: batch index bits [src, src+len) -> physical dst
  int nruns = 0;
  uint8_t run_src[16], run_len[16], run_dst[16];
  // every phase's map in program order: maps[0] = load map, maps[i] = the
  // target of the i-th PK_XCHG (the last one is the store map)
  std::vector<PhaseMap> maps;
  int act[kMaxPhasedM];      // physical qubit of local bit j
  int jit_module = -1;       // index of the JIT module holding this kernel, -1: none
  // launch shape of the specialised kernel (set by jit_source): dynamic
  // shared memory in bytes, the CTAs per SM its launch bounds ask for, and
  // its batch-load form (0 direct loads, 1 cp.async prefetch into a separate
  // staging buffer, 2 prefetch into the exchange tile after the last exchange)
  int jit_smem = 0;
  int jit_min_blocks = 1;
  int jit_prefetch = 0;
};

// Padded shared-memory layout of the JIT kernels: one spare amplitude per 16,
// 256 and 4096.  Additive over disjoint bit sets, so an address is a thread
// part plus a compile-time register part; distinct residues mod 4 of the
// four half-warp lane bits give distinct banks.
inline uint32_t pad_index(uint32_t li) { return li + (li >> 4) + (li >> 8) + (li >> 12); }
inline uint32_t pad_size(int m) { return pad_index((1u << m) - 1u) + 1u; }

}  // namespace qs
