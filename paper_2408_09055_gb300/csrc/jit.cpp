// Plan-time specialisation of shared-memory kernels (kernel type 2 of the
// paper's "Cost Function in Kernelize"; insular handling of Appendix A.2).
//
// Each register-phased program (shm_program.cpp) is turned into one
// straight-line CUDA kernel and compiled for sm_103a with NVRTC:
//  * every register bit, thread bit, matrix entry and HBM/shared-memory
//    offset is a compile-time constant, so the interpreter's dispatch,
//    control masks and runtime address arithmetic disappear;
//  * X, CX on register bits and SWAP become register renames (no code);
//  * zero and unit terms of every 2x2 and diagonal factor are dropped;
//  * the exchange tile uses the padded layout pad_index(), which is
//    additive, so each shared access is `tile[thread_offset + constant]`.
// Kernels are compiled in parallel batches; the cubins are cached on disk
// keyed by a hash of the source.
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cinttypes>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>
#include <sys/stat.h>
#include <thread>
#include <unistd.h>

#include "internal.hpp"
#include "shm_program.hpp"

namespace qs {

namespace {

std::string flit(float v) {
  char b[48];
  std::snprintf(b, sizeof b, "%.9ef", (double)v);
  return b;
}

float word_f(uint32_t w) {
  float f;
  std::memcpy(&f, &w, 4);
  return f;
}

// One real component of a sum of products: terms (coef, operand).
std::string lin(const std::vector<std::pair<float, std::string>>& terms) {
  std::string acc;
  for (const auto& t : terms) {
    float c = t.first;
    if (c == 0.0f) continue;
    if (acc.empty()) {
      if (c == 1.0f) acc = t.second;
      else if (c == -1.0f) acc = "(-" + t.second + ")";
      else acc = "(" + flit(c) + "*" + t.second + ")";
    } else {
      if (c == 1.0f) acc = "(" + acc + "+" + t.second + ")";
      else if (c == -1.0f) acc = "(" + acc + "-" + t.second + ")";
      else acc = "fmaf(" + flit(c) + "," + t.second + "," + acc + ")";
    }
  }
  return acc.empty() ? std::string("0.0f") : acc;
}

// One real component of a sum of products whose coefficients are either
// constants (c, a empty) or per-thread values (the expression a, added with
// the sign of c = +-1).
struct LT {
  float c;
  std::string a, x;
};
std::string lin_rt(const std::vector<LT>& terms) {
  std::string acc;
  for (const LT& t : terms) {
    if (t.a.empty()) {
      const float c = t.c;
      if (c == 0.0f) continue;
      if (acc.empty()) {
        if (c == 1.0f) acc = t.x;
        else if (c == -1.0f) acc = "(-" + t.x + ")";
        else acc = "(" + flit(c) + "*" + t.x + ")";
      } else {
        if (c == 1.0f) acc = "(" + acc + "+" + t.x + ")";
        else if (c == -1.0f) acc = "(" + acc + "-" + t.x + ")";
        else acc = "fmaf(" + flit(c) + "," + t.x + "," + acc + ")";
      }
    } else {
      const std::string c = t.c < 0 ? "(-" + t.a + ")" : t.a;
      acc = acc.empty() ? "(" + c + "*" + t.x + ")" : "fmaf(" + c + "," + t.x + "," + acc + ")";
    }
  }
  return acc.empty() ? std::string("0.0f") : acc;
}

struct CF {
  float re, im;
};

// re/im parts of sum_c u_c * v_c for complex constants u_c and variables v_c
std::string cre(const std::vector<std::pair<CF, std::string>>& t) {
  std::vector<std::pair<float, std::string>> r;
  for (auto& x : t) {
    r.push_back({x.first.re, x.second + ".x"});
    r.push_back({-x.first.im, x.second + ".y"});
  }
  return lin(r);
}
std::string cim(const std::vector<std::pair<CF, std::string>>& t) {
  std::vector<std::pair<float, std::string>> r;
  for (auto& x : t) {
    r.push_back({x.first.re, x.second + ".y"});
    r.push_back({x.first.im, x.second + ".x"});
  }
  return lin(r);
}

bool unit(CF c) { return c.re == 1.0f && c.im == 0.0f; }

using cd = std::complex<double>;

struct Gen {
  const ShmProgramV2& pg;
  std::ostringstream o;
  int nm[kRegAmps];  // register index j -> variable r<nm[j]>
  int phase = 0;
  std::string after_last_xchg;  // emitted once the last exchange has read the tile
  // Deferred factors: variable r<v> holds its amplitude divided by pend[v].
  // A diagonal factor on register bits only multiplies pend (no code).  A
  // dense 2x2 or 4x4 product folds its inputs' factors into its constants
  // and, when a later dense product of the same phase reads the output,
  // divides the output row by its largest coefficient and keeps that
  // coefficient in pend, so that term costs an add instead of a complex
  // multiply.  Exchanges, the store and ops under a runtime condition
  // first apply what is pending (one complex multiply per variable whose
  // factor is not 1).  Scaling a row by one of its own coefficients leaves
  // its rounding error bound unchanged.
  bool defer = false;
  bool dry = false;           // lookahead pass: records which outputs are read again
  std::vector<char> consumed;  // per dense output, in order
  int out_id = 0;
  int last_out[kRegAmps];
  cd pend[kRegAmps];
  // Runtime factors: a diagonal factor under a runtime condition (a control
  // or phase on a thread or batch bit) becomes a per-thread select instead
  // of a branch when the lookahead pass has seen a later dense product of
  // the same phase read every variable it touches; rtf[v] then names the
  // per-thread float2 by which r<v> must still be multiplied, and the
  // product takes it into its coefficients (one complex product per
  // coefficient and thread, not per amplitude).
  std::string rtf[kRegAmps];
  int nfac = 0;
  std::map<std::string, std::string> fac_memo;  // expression -> declared factor variable
  int rt_id = 0;                                // runtime diagonal ops, in order
  std::vector<int> rt_open;                     // lookahead: variables of op id not yet read by a product
  std::vector<int> rt_pend[kRegAmps];           // lookahead: op ids whose factor variable w still carries
  std::vector<char> rt_ok;                      // op id may be deferred
  bool rt_defer = false;
  explicit Gen(const ShmProgramV2& p) : pg(p) {
    for (int j = 0; j < kRegAmps; ++j) {
      nm[j] = j;
      last_out[j] = -1;
      pend[j] = 1.0;
    }
  }
  std::string v(int j) const { return "r" + std::to_string(nm[j]); }

  static CF cf_of(cd z) { return CF{(float)z.real(), (float)z.imag()}; }
  static std::string cconst(CF c) { return "make_float2(" + flit(c.re) + "," + flit(c.im) + ")"; }

  // a per-thread float2 holding `expr`, declared once in the batch loop
  std::string fac(const std::string& expr) {
    auto it = fac_memo.find(expr);
    if (it != fac_memo.end()) return it->second;
    const std::string name = "f" + std::to_string(nfac++);
    o << "const float2 " << name << "=" << expr << ";\n";
    fac_memo.emplace(expr, name);
    return name;
  }
  // runtime factor f times the constant c
  std::string fac_times(const std::string& f, CF c) {
    if (unit(c)) return f;
    return fac("make_float2(" + lin({{c.re, f + ".x"}, {-c.im, f + ".y"}}) + "," +
               lin({{c.re, f + ".y"}, {c.im, f + ".x"}}) + ")");
  }
  void compose(int w, const std::string& f) {
    if (rtf[w].empty()) rtf[w] = f;
    else rtf[w] = fac("make_float2(" + rtf[w] + ".x*" + f + ".x-" + rtf[w] + ".y*" + f + ".y," + rtf[w] + ".x*" + f +
                      ".y+" + rtf[w] + ".y*" + f + ".x)");
  }

  // Whether the next runtime diagonal op (touching registers with bit A =
  // 0 and/or 1; A < 0: every register) is deferred.  The lookahead pass
  // records the variables it touches; the real pass defers it when a dense
  // product of the same phase read all of them before any flush.
  bool runtime_diag(bool t0, bool t1, int A) {
    if (!defer || !rt_defer) return false;
    const int id = rt_id++;
    if (dry) {
      int cnt = 0;
      for (int j = 0; j < kRegAmps; ++j)
        if (A < 0 ? (t0 || t1) : (((j >> A) & 1) ? t1 : t0)) {
          rt_pend[nm[j]].push_back(id);
          ++cnt;
        }
      rt_open.push_back(cnt);
      return false;
    }
    return id < (int)rt_ok.size() && rt_ok[id];
  }

  // applies variable w's pending factors
  void flush_var(int w) {
    last_out[w] = -1;
    rt_pend[w].clear();
    const CF e = cf_of(pend[w]);
    pend[w] = 1.0;
    const std::string x = "r" + std::to_string(w);
    if (!rtf[w].empty()) {
      const std::string c = fac_times(rtf[w], e);
      rtf[w].clear();
      o << "{const float2 x=" << x << ";" << x << "=make_float2(" << c << ".x*x.x-" << c << ".y*x.y," << c
        << ".x*x.y+" << c << ".y*x.x);}\n";
      return;
    }
    if (unit(e)) return;
    o << "{const float2 x=" << x << ";" << x << "=make_float2(" << cre({{e, "x"}}) << "," << cim({{e, "x"}})
      << ");}\n";
  }
  void flush_all() {
    for (int w = 0; w < kRegAmps; ++w) flush_var(w);
  }

  void diag(int j, CF e) {  // r_j *= e, a factor known at generation time
    if (defer) pend[nm[j]] *= cd(e.re, e.im);
    else mulc(j, e);
  }

  // r_idx[i] <- sum_k M[s*i + k] r_idx[k] for one group of s = 2 or 4
  // registers; `cond`: the code sits under a runtime condition (the group's
  // pending factors were applied before it, and its outputs keep factor 1)
  void dense(const int* idx, int s, const CF* M, bool cond) {
    int w[4];
    for (int k = 0; k < s; ++k) w[k] = nm[idx[k]];
    cd E[16];
    for (int i = 0; i < s; ++i)
      for (int k = 0; k < s; ++k) E[s * i + k] = cd(M[s * i + k].re, M[s * i + k].im) * pend[w[k]];
    if (defer && !cond)
      for (int k = 0; k < s; ++k) {
        if (last_out[w[k]] >= 0) consumed[last_out[w[k]]] = 1;
        for (int id : rt_pend[w[k]]) --rt_open[id];
        rt_pend[w[k]].clear();
      }
    cd d[4];
    int piv[4];
    for (int i = 0; i < s; ++i) {
      d[i] = 1.0;
      piv[i] = -1;
      if (!defer || cond) continue;
      const int id = out_id++;
      if (dry) consumed.push_back(0);
      else if (id < (int)consumed.size() && consumed[id]) {
        int kb = -1;  // the pivot: the largest coefficient known at generation time
        for (int k = 0; k < s; ++k)
          if (rtf[w[k]].empty() && (kb < 0 || std::abs(E[s * i + k]) > std::abs(E[s * i + kb]))) kb = k;
        if (kb >= 0 && std::abs(E[s * i + kb]) > 1e-30) {
          d[i] = E[s * i + kb];
          piv[i] = kb;
        }
      }
    }
    // coefficients that carry an input's runtime factor, declared before the block
    std::string rc[16];
    for (int i = 0; i < s; ++i)
      for (int k = 0; k < s; ++k) {
        const CF c = cf_of(E[s * i + k] / d[i]);
        if (!rtf[w[k]].empty() && !(c.re == 0.0f && c.im == 0.0f)) rc[s * i + k] = fac_times(rtf[w[k]], c);
      }
    o << "{const float2 ";
    for (int k = 0; k < s; ++k) o << (k ? "," : "") << "x" << k << "=" << v(idx[k]);
    o << ";\n";
    for (int i = 0; i < s; ++i) {
      std::vector<LT> re, im;
      auto term = [&](int k) {
        const std::string x = "x" + std::to_string(k);
        if (!rc[s * i + k].empty()) {  // runtime coefficient c: (c.x xr - c.y xi, c.x xi + c.y xr)
          const std::string& c = rc[s * i + k];
          re.push_back({1.0f, c + ".x", x + ".x"});
          re.push_back({-1.0f, c + ".y", x + ".y"});
          im.push_back({1.0f, c + ".x", x + ".y"});
          im.push_back({1.0f, c + ".y", x + ".x"});
          return;
        }
        const CF c = k == piv[i] ? CF{1.0f, 0.0f} : cf_of(E[s * i + k] / d[i]);
        re.push_back({c.re, "", x + ".x"});
        re.push_back({-c.im, "", x + ".y"});
        im.push_back({c.re, "", x + ".y"});
        im.push_back({c.im, "", x + ".x"});
      };
      if (piv[i] >= 0) term(piv[i]);
      for (int k = 0; k < s; ++k)
        if (k != piv[i]) term(k);
      o << v(idx[i]) << "=make_float2(" << lin_rt(re) << "," << lin_rt(im) << ");\n";
    }
    o << "}\n";
    for (int i = 0; i < s; ++i) {
      pend[w[i]] = d[i];
      if (!cond) rtf[w[i]].clear();
      if (defer && !cond) last_out[w[i]] = out_id - s + i;
    }
  }

  // value (0/1) of a qubit reference that is not a register slot
  std::string known(uint32_t ref) const {
    if (ref & REF_GLOBAL) return "((unsigned)((base | hi) >> " + std::to_string(ref & 63u) + ") & 1u)";
    const PhaseMap& pm = pg.maps[phase];
    int b = (int)(ref & 31u);
    for (int k = 0; k < pm.nt; ++k)
      if (pm.T[k] == b) return "((tid >> " + std::to_string(k) + ") & 1u)";
    return "0u";  // unreachable for a well-formed program
  }

  void mulc(int j, CF e) {  // r_j *= e
    if (unit(e)) return;
    std::string x = v(j);
    o << "{const float2 x=" << x << ";" << x << "=make_float2(" << cre({{e, "x"}}) << ","
      << cim({{e, "x"}}) << ");}\n";
  }

  void g1(int t, CF u00, CF u01, CF u10, CF u11, bool cond = false) {
    const CF M[4] = {u00, u01, u10, u11};
    for (int j = 0; j < kRegAmps; ++j) {
      if (j & (1 << t)) continue;
      const int idx[2] = {j, j | (1 << t)};
      dense(idx, 2, M, cond);
    }
  }

  void swap_pair(int j, int k) { std::swap(nm[j], nm[k]); }

  void xchg(const PhaseMap& next, int next_index) {
    flush_all();
    o << "__syncthreads();\n";
    const PhaseMap& cur = pg.maps[phase];
    for (int j = 0; j < kRegAmps; ++j) {
      uint32_t li = 0;
      for (int i = 0; i < kRegBits; ++i)
        if ((j >> i) & 1) li |= 1u << cur.R[i];
      o << "tile[sp" << phase << "+" << pad_index(li) << "u]=" << v(j) << ";\n";
    }
    o << "__syncthreads();\n";
    for (int j = 0; j < kRegAmps; ++j) {
      nm[j] = j;
      uint32_t li = 0;
      for (int i = 0; i < kRegBits; ++i)
        if ((j >> i) & 1) li |= 1u << next.R[i];
      o << v(j) << "=tile[sp" << next_index << "+" << pad_index(li) << "u];\n";
    }
    phase = next_index;
    if (next_index == (int)pg.maps.size() - 1) o << after_last_xchg;
  }

  bool body() {
    const std::vector<uint32_t>& w = pg.prog;
    size_t pc = 0;
    int xchg_seen = 0;
    auto cf = [&](size_t at) { return CF{word_f(w[at]), word_f(w[at + 1])}; };
    while (pc < w.size()) {
      const uint32_t op = w[pc] & 0xFFu, A = (w[pc] >> 8) & 0xFFu, B = (w[pc] >> 16) & 0xFFu,
                     Cu = w[pc] >> 24;
      switch (op) {
        case PK_END:
          return true;
        case PK_G1:
          g1((int)A, cf(pc + 1), cf(pc + 3), cf(pc + 5), cf(pc + 7));
          pc += 9;
          break;
        case PK_G1R:
          g1((int)A, CF{word_f(w[pc + 1]), 0}, CF{word_f(w[pc + 2]), 0}, CF{word_f(w[pc + 3]), 0},
             CF{word_f(w[pc + 4]), 0});
          pc += 5;
          break;
        case PK_G1X:
          g1((int)A, CF{word_f(w[pc + 1]), 0}, CF{0, word_f(w[pc + 2])}, CF{0, word_f(w[pc + 3])},
             CF{word_f(w[pc + 4]), 0});
          pc += 5;
          break;
        case PK_G1C: {
          CF u00 = cf(pc + 1), u01 = cf(pc + 3), u10 = cf(pc + 5), u11 = cf(pc + 7);
          if (B < (uint32_t)kRegBits) {
            const CF M[4] = {u00, u01, u10, u11};
            for (int j = 0; j < kRegAmps; ++j) {
              if ((j & (1 << A)) || !((j >> B) & 1)) continue;
              const int idx[2] = {j, j | (1 << A)};
              dense(idx, 2, M, false);
            }
          } else {
            for (int j = 0; j < kRegAmps; ++j) flush_var(nm[j]);
            o << "if (" << known(B) << ") {\n";
            g1((int)A, u00, u01, u10, u11, true);
            o << "}\n";
          }
          pc += 9;
          break;
        }
        case PK_XG:
          for (int j = 0; j < kRegAmps; ++j)
            if (!(j & (1 << A))) swap_pair(j, j | (1 << A));
          pc += 1;
          break;
        case PK_XGS:
          for (int j = 0; j < kRegAmps; ++j)
            if (!(j & (1 << A)) && ((j >> B) & 1)) swap_pair(j, j | (1 << A));
          pc += 1;
          break;
        case PK_XGK:
          for (int j = 0; j < kRegAmps; ++j) flush_var(nm[j]);
          o << "if (" << known(B) << ") {\n";
          for (int j = 0; j < kRegAmps; ++j)
            if (!(j & (1 << A))) {
              std::string a = v(j), b = v(j | (1 << A));
              o << "{const float2 x=" << a << ";" << a << "=" << b << ";" << b << "=x;}\n";
            }
          o << "}\n";
          pc += 1;
          break;
        case PK_D1B: {
          CF e = cf(pc + 1);
          for (int j = 0; j < kRegAmps; ++j)
            if (j & (1 << A)) diag(j, e);
          pc += 3;
          break;
        }
        case PK_D1: {
          CF e0 = cf(pc + 1), e1 = cf(pc + 3);
          for (int j = 0; j < kRegAmps; ++j) diag(j, (j & (1 << A)) ? e1 : e0);
          pc += 5;
          break;
        }
        case PK_D1K: {
          CF d[4] = {cf(pc + 1), cf(pc + 3), cf(pc + 5), cf(pc + 7)};
          // register j takes d[2 kb + bit A of j], kb the known bit's value
          bool touch[2];
          for (int a = 0; a < 2; ++a) touch[a] = !(unit(d[a]) && unit(d[2 + a]));
          if (runtime_diag(touch[0], touch[1], (int)A)) {
            std::string f[2];
            for (int a = 0; a < 2; ++a)
              if (touch[a]) f[a] = fac("(" + known(B) + " ? " + cconst(d[2 + a]) + " : " + cconst(d[a]) + ")");
            for (int j = 0; j < kRegAmps; ++j)
              if (touch[(j >> A) & 1]) compose(nm[j], f[(j >> A) & 1]);
          } else {
            for (int kb = 0; kb < 2; ++kb) {
              if (unit(d[2 * kb]) && unit(d[2 * kb + 1])) continue;
              o << "if (" << known(B) << (kb ? "" : " == 0u") << ") {\n";
              for (int j = 0; j < kRegAmps; ++j) mulc(j, d[2 * kb + ((j >> A) & 1)]);
              o << "}\n";
            }
          }
          pc += 9;
          break;
        }
        case PK_D2: {
          CF d[4] = {cf(pc + 1), cf(pc + 3), cf(pc + 5), cf(pc + 7)};
          for (int j = 0; j < kRegAmps; ++j) diag(j, d[((j >> A) & 1) | (((j >> B) & 1) << 1)]);
          pc += 9;
          break;
        }
        case PK_D2P: {
          CF e = cf(pc + 1);
          for (int j = 0; j < kRegAmps; ++j)
            if (((j >> A) & 1) && ((j >> B) & 1)) diag(j, e);
          pc += 3;
          break;
        }
        case PK_D0: {
          CF d[4] = {cf(pc + 1), cf(pc + 3), cf(pc + 5), cf(pc + 7)};
          std::string k0 = known(A), k1 = (B == REF_NONE) ? std::string("0u") : known(B);
          bool any = false;  // a factor other than 1 for some value of the known bits
          for (int idx = 0; idx < 4; ++idx)
            if (!((Cu >> idx) & 1u) && !(B == REF_NONE && idx >= 2) && !unit(d[idx])) any = true;
          if (any && runtime_diag(true, true, -1)) {
            auto val = [&](int idx) { return ((Cu >> idx) & 1u) ? std::string("make_float2(1.0f,0.0f)") : cconst(d[idx]); };
            std::string e = "(" + k0 + " ? " + val(1) + " : " + val(0) + ")";
            if (B != REF_NONE) e = "(" + k1 + " ? (" + k0 + " ? " + val(3) + " : " + val(2) + ") : " + e + ")";
            const std::string f = fac(e);
            for (int j = 0; j < kRegAmps; ++j) compose(nm[j], f);
            pc += 9;
            break;
          }
          for (int idx = 0; idx < 4; ++idx) {
            if ((Cu >> idx) & 1u) continue;
            if (B == REF_NONE && idx >= 2) continue;
            o << "if (" << k0 << " == " << (idx & 1) << "u && " << k1 << " == " << (idx >> 1)
              << "u) {\n";
            for (int j = 0; j < kRegAmps; ++j) mulc(j, d[idx]);
            o << "}\n";
          }
          pc += 9;
          break;
        }
        case PK_SWAPR:
          for (int j = 0; j < kRegAmps; ++j)
            if (((j >> A) & 1) && !((j >> B) & 1)) swap_pair(j, j ^ (1 << A) ^ (1 << B));
          pc += 1;
          break;
        case PK_XX: {
          float c = word_f(w[pc + 1]), s = word_f(w[pc + 2]);
          const CF M[4] = {CF{c, 0}, CF{0, -s}, CF{0, -s}, CF{c, 0}};
          for (int j = 0; j < kRegAmps; ++j) {
            if ((j >> B) & 1) continue;
            const int idx[2] = {j, j ^ (1 << A) ^ (1 << B)};
            dense(idx, 2, M, false);
          }
          pc += 3;
          break;
        }
        case PK_SCALE: {
          CF e = cf(pc + 1);
          for (int j = 0; j < kRegAmps; ++j) diag(j, e);
          pc += 3;
          break;
        }
        case PK_G2: {  // dense 4x4 on slots A < B
          CF g[16];
          for (int e = 0; e < 16; ++e) g[e] = cf(pc + 1 + 2 * e);
          for (int j = 0; j < kRegAmps; ++j) {
            if (((j >> A) & 1) || ((j >> B) & 1)) continue;
            const int idx[4] = {j, j | (1 << A), j | (1 << B), j | (1 << A) | (1 << B)};
            dense(idx, 4, g, false);
          }
          pc += 33;
          break;
        }
        case PK_XCHG:
          ++xchg_seen;
          if (xchg_seen >= (int)pg.maps.size()) return false;
          xchg(pg.maps[xchg_seen], xchg_seen);
          pc += 1 + kRegBits + A;
          break;
        default:
          return false;
      }
    }
    return false;
  }
};

std::string thread_expr(const PhaseMap& pm, const uint64_t* value_of_local) {
  std::ostringstream e;
  e << "0u";
  for (int k = 0; k < pm.nt; ++k) {
    uint64_t val = value_of_local[pm.T[k]];
    e << " + (((tid >> " << k << ") & 1u) * " << val << "u)";
  }
  return e.str();
}

}  // namespace

// Batch-load form of a specialised kernel: QSIM_JIT_PREFETCH = 0, 1 or 2
// overrides the default, 0.  Measured on the 30-qubit mixed circuit (|A| <=
// 12): loads straight into registers 3.40 ms per launch; a cp.async prefetch
// of the next batch into a separate staging buffer 4.27 ms (3 instead of 4
// CTAs per SM); the prefetch into the exchange tile after the last exchange
// 3.47 ms.
static int prefetch_form() {
  const char* e = std::getenv("QSIM_JIT_PREFETCH");
  if (e && (e[0] == '0' || e[0] == '1' || e[0] == '2') && !e[1]) return e[0] - '0';
  return 0;
}

// Deferred factors in the generated code (Gen::defer): QSIM_JIT_DEFER = 0
// turns them off, 1 (the default) keeps the factors known at generation
// time, 2 also defers runtime-conditioned diagonals (Gen::rt_defer).
// Measured at 30 qubits (plan A, one process): mixed circuit 491.5 ms at
// level 1, 495.9 ms at level 2; entangling circuit 322 and 365 ms.  Level 2
// keeps per-thread factors and coefficients live across the phase, and
// under the 128-register bound of four CTAs per SM the entangling kernels
// spill (ptxas: 164-316 bytes of spill stores per thread against none).
static int defer_factors() {
  const char* e = std::getenv("QSIM_JIT_DEFER");
  if (e && (e[0] == '0' || e[0] == '1' || e[0] == '2') && !e[1]) return e[0] - '0';
  return 1;
}

void jit_shape(const ShmProgramV2& pg, int* form, int* smem, int* min_blocks) {
  const int m = pg.m;
  const bool xch = pg.maps.size() > 1;
  const size_t tile = sizeof(float) * 2 * pad_size(m), stg = sizeof(float) * 2 << m;
  const int f = prefetch_form();
  size_t bytes;
  if (f == 0) bytes = tile;                       // loads straight into registers
  else if (f == 1) bytes = (xch ? tile : 0) + stg;  // staging beside the exchange tile
  else bytes = xch ? tile : stg;                  // staging inside the exchange tile
  // CTAs per SM: what shared memory allows (227 KiB, 1 KiB reserved per
  // CTA), at most 2^(14-m) so that a thread keeps >= 128 registers
  int mb = 1 << (kMaxShmActive - m);
  if (f != 0) mb = std::max(1, std::min(mb, (int)((227u << 10) / (bytes + 1024))));
  *form = f;
  *smem = (int)bytes;
  *min_blocks = mb;
}

bool jit_source(const ShmProgramV2& pg, int n, const std::string& name, std::string* out) {
  const int m = pg.m;
  const int nt = m - kRegBits;
  const unsigned nthr = 1u << nt;
  Gen g(pg);
  std::ostringstream& o = g.o;
  uint64_t phys[kMaxShmActive], padv[kMaxShmActive];
  for (int j = 0; j < m; ++j) {
    phys[j] = 1ull << pg.act[j];
    padv[j] = pad_index(1u << j);
    if (pg.act[j] >= 32) return false;
  }
  int form = 0, smem = 0, minb = 1;
  jit_shape(pg, &form, &smem, &minb);
  const bool xch = pg.maps.size() > 1;
  uint64_t ld_off[kRegAmps];
  {
    const PhaseMap& lm = pg.maps.front();
    for (int j = 0; j < kRegAmps; ++j) {
      ld_off[j] = 0;
      for (int i = 0; i < kRegBits; ++i)
        if ((j >> i) & 1) ld_off[j] |= phys[lm.R[i]];
    }
  }
  // the batch's base address: batch index bits spread over the non-active qubits
  o << "static __device__ __forceinline__ unsigned long long " << name
    << "_base(unsigned long long bt) {\nreturn 0ull";
  for (int r = 0; r < pg.nruns; ++r)
    o << " | (((bt >> " << (int)pg.run_src[r] << ") & " << ((1ull << pg.run_len[r]) - 1) << "ull) << "
      << (int)pg.run_dst[r] << ")";
  o << ";\n}\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << nthr << ", " << minb << ")\n"
    << name << "(float2* __restrict__ psi, unsigned long long nb, unsigned long long hi) {\n"
    << "extern __shared__ float2 tile[];\n"
    << "const unsigned tid = threadIdx.x;\n";
  o << "const unsigned ptl = " << thread_expr(pg.maps.front(), phys) << ";\n";
  o << "const unsigned pts = " << thread_expr(pg.maps.back(), phys) << ";\n";
  for (size_t p = 0; p < pg.maps.size(); ++p)
    o << "const unsigned sp" << p << " = " << thread_expr(pg.maps[p], padv) << ";\n";
  std::string issue;  // prefetch of batch bt + gridDim.x into this thread's staging slots
  if (form != 0) {
    // staging slot of register j of thread t: float2 index j * nthr + t
    // (consecutive lanes, consecutive 8-byte words: no bank conflicts)
    const uint32_t stg0 = (form == 1 && xch) ? pad_size(m) : 0;
    o << "float2* const stg = tile + " << stg0 << "u;\n";
    o << "unsigned ss;\nasm(\"{.reg .u64 t; cvta.to.shared.u64 t, %1; cvt.u32.u64 %0, t;}\" : \"=r\"(ss) : "
         "\"l\"(stg + tid));\n";
    std::ostringstream is;
    is << "{\nconst unsigned long long nbt = bt + gridDim.x;\nif (nbt < nb) {\n"
       << "unsigned long long gp;\nasm(\"cvta.to.global.u64 %0, %1;\" : \"=l\"(gp) : \"l\"(psi + (" << name
       << "_base(nbt) | ptl)));\n";
    for (int j = 0; j < kRegAmps; ++j)
      is << "asm volatile(\"cp.async.ca.shared.global [%0+" << (8u * nthr * (uint32_t)j) << "], [%1+"
         << (8ull * ld_off[j]) << "], 8;\" :: \"r\"(ss), \"l\"(gp) : \"memory\");\n";
    is << "}\nasm volatile(\"cp.async.commit_group;\" ::: \"memory\");\n}\n";
    issue = is.str();
    // the first batch: nothing else uses the staging slots yet
    o << "{\nconst unsigned long long bt = (unsigned long long)blockIdx.x - gridDim.x;\n" << issue << "}\n";
  }
  o << "for (unsigned long long bt = blockIdx.x; bt < nb; bt += gridDim.x) {\n";
  o << "const unsigned long long base = " << name << "_base(bt);\n";
  if (form == 0) {
    o << "const float2* __restrict__ ip = psi + (base | ptl);\n";
    for (int j = 0; j < kRegAmps; ++j) o << "float2 r" << j << " = ip[" << ld_off[j] << "u];\n";
  } else {
    o << "asm volatile(\"cp.async.wait_group 0;\" ::: \"memory\");\n";
    for (int j = 0; j < kRegAmps; ++j) o << "float2 r" << j << " = stg[" << (nthr * (uint32_t)j) << "u + tid];\n";
    if (form == 1 || !xch) {
      o << issue;  // own slots only: read above, refilled now
    } else {
      // the exchange tile holds the slots: refill once every thread has read
      // the last exchange's values
      g.after_last_xchg = "__syncthreads();\n" + issue;
    }
  }
  if (const int level = defer_factors()) {
    Gen look(pg);  // the lookahead pass: which dense outputs are read again
    look.defer = look.dry = true;
    look.rt_defer = g.rt_defer = level >= 2;
    if (!look.body()) return false;
    g.defer = true;
    g.consumed = std::move(look.consumed);
    for (int c : look.rt_open) g.rt_ok.push_back(c == 0);
  }
  if (!g.body()) return false;
  if (g.phase != (int)pg.maps.size() - 1) return false;
  g.flush_all();
  o << "float2* __restrict__ op = psi + (base | pts);\n";
  {
    const PhaseMap& sm = pg.maps.back();
    for (int j = 0; j < kRegAmps; ++j) {
      uint64_t off = 0;
      for (int i = 0; i < kRegBits; ++i)
        if ((j >> i) & 1) off |= phys[sm.R[i]];
      o << "op[" << off << "u] = " << g.v(j) << ";\n";
    }
  }
  o << "}\n}\n";
  (void)n;
  *out = o.str();
  return true;
}

// ---- NVRTC -----------------------------------------------------------------------

static uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

static std::string cache_dir() {
  const char* e = std::getenv("QSIM_JIT_CACHE");
  if (e && *e) return e;
  const char* home = std::getenv("HOME");
  std::string d = std::string(home && *home ? home : "/tmp") + "/.cache/qsim-jit";
  return d;
}

static void mkdirs(const std::string& d) {
  std::string cur;
  for (size_t i = 0; i < d.size(); ++i) {
    cur += d[i];
    if (d[i] == '/' && cur.size() > 1) mkdir(cur.c_str(), 0755);
  }
  mkdir(d.c_str(), 0755);
}

static bool compile_one(const std::string& src, std::vector<char>* cubin, std::string* log) {
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo"};
  // the cache name: two independent hashes of the source and the options,
  // and the source length, so that no other program maps to the same file
  std::string keyed = src;
  for (const char* o : opts) (keyed += '\n') += o;
  const std::string dir = cache_dir();
  char key[80];
  std::snprintf(key, sizeof key, "%016" PRIx64 "%016zx-%zu", fnv1a(keyed), std::hash<std::string>{}(keyed),
                src.size());
  const std::string path = dir + "/" + key + ".cubin";
  {
    std::ifstream f(path, std::ios::binary);
    if (f) {
      cubin->assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
      if (!cubin->empty()) return true;
    }
  }
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "qsim_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return false;
  nvrtcResult r = nvrtcCompileProgram(prog, (int)(sizeof opts / sizeof opts[0]), opts);
  if (r != NVRTC_SUCCESS) {
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    log->resize(ls);
    nvrtcGetProgramLog(prog, log->data());
    nvrtcDestroyProgram(&prog);
    return false;
  }
  size_t sz = 0;
  nvrtcGetCUBINSize(prog, &sz);
  cubin->resize(sz);
  nvrtcGetCUBIN(prog, cubin->data());
  nvrtcDestroyProgram(&prog);
  mkdirs(dir);
  // a name no other thread or process writes (several ranks may compile the
  // same plan at once); the rename publishes the file atomically
  static std::atomic<unsigned> seq{0};
  const std::string tmp = path + ".tmp." + std::to_string((long long)getpid()) + "." +
                          std::to_string((unsigned long long)std::hash<std::thread::id>{}(std::this_thread::get_id())) +
                          "." + std::to_string(seq.fetch_add(1));
  {
    std::ofstream f(tmp, std::ios::binary);
    f.write(cubin->data(), (std::streamsize)cubin->size());
  }
  std::rename(tmp.c_str(), path.c_str());
  return true;
}

// Compiles every phased program of the plan into cubins (one module per
// batch of kernels), in parallel.  Programs that fail keep the interpreter.
int jit_compile_plan(PlanImpl* p) {
  std::vector<int> idx;
  for (size_t i = 0; i < p->shm2.size(); ++i)
    if (p->shm2[i].ok) idx.push_back((int)i);
  p->jit_modules.clear();
  if (idx.empty()) return QS_OK;
  // modules of at most ~64 KB of source (a large kernel gets its own module):
  // front-end and ptxas time grow faster than linearly with module size, and
  // more modules spread over more threads
  const size_t budget = 64 * 1024;
  std::vector<std::string> srcs;
  std::vector<std::vector<int>> members;
  for (int i : idx) {
    std::string name = "qsk" + std::to_string(i), s;
    ShmProgramV2& pg = p->shm2[i];
    jit_shape(pg, &pg.jit_prefetch, &pg.jit_smem, &pg.jit_min_blocks);
    if (!jit_source(pg, p->n, name, &s)) continue;
    if (srcs.empty() || srcs.back().size() + s.size() > budget) {
      srcs.emplace_back();
      members.emplace_back();
    }
    srcs.back() += s;
    members.back().push_back(i);
  }
  const int nmod = (int)srcs.size();
  p->jit_modules.assign(nmod, std::vector<char>());
  std::vector<char> ok(nmod, 0);
  std::atomic<int> next{0};
  std::string first_log;
  std::mutex log_mu;
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  unsigned nth = std::min<unsigned>(hw, (unsigned)nmod);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nth; ++t)
    th.emplace_back([&]() {
      for (int k; (k = next.fetch_add(1)) < nmod;) {
        if (srcs[k].empty()) continue;
        std::string log;
        ok[k] = compile_one(srcs[k], &p->jit_modules[k], &log);
        if (!ok[k]) {
          std::lock_guard<std::mutex> lk(log_mu);
          if (first_log.empty()) first_log = log;
        }
      }
    });
  for (auto& t : th) t.join();
  for (int k = 0; k < nmod; ++k)
    for (int i : members[k]) {
      p->shm2[i].jit_module = ok[k] ? k : -1;
    }
  p->jit_log = first_log;
  return QS_OK;
}

}  // namespace qs
