// Device scalar expressions: the C-ABI counterpart of the managed-memory
// expression templates and Eval() of Sec. 3.2.1.
//
// C++ expression templates cannot cross a C ABI, so an expression arrives as
// a postfix list of terms (managed scalars, constants, operators).  Creating
// the expression "freezes" it (Eval): the list becomes a DAG in which equal
// subexpressions are one node (common-subexpression elimination), subtrees of
// constants are folded where the host computes exactly what the device would
// (the correctly rounded + - * / sqrt, and neg, abs, min, max), and a few
// rewrites that never change a value are applied (x * 1, x / 1, x - 0,
// -(-x)).  The frozen program is a list of SSA instructions; executing it is
// one kernel launch, marked as reading every input scalar and writing the
// output (Sec. 3.1.2).  A consumer kernel can also evaluate the program in its
// own prologue (apcg_vec_axpy_expr_async), so the scalar never needs a
// launch of its own -- the fusion of scalar work into its consumers that the
// CG kernels of this library use throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "apcg_internal.hpp"

namespace apcg {
namespace {

constexpr int kMaxIns = 64;    // instructions of a frozen program
constexpr int kMaxLoads = 16;  // distinct input scalars

struct Ins {
  uint8_t op;  // apcg_expr_op
  uint8_t a, b;  // operand instructions
  uint8_t load;  // APCG_EX_SCALAR: index into the loads
  int32_t pad;
  double c;  // APCG_EX_CONST
};

struct Prog {
  int32_t n = 0;      // instructions; the result is instruction n - 1
  int32_t nload = 0;
  Ins ins[kMaxIns];
  const double* loads[kMaxLoads];
};

__device__ __forceinline__ double eval_prog(const Prog& P) {
  double r[kMaxIns];
  for (int i = 0; i < P.n; ++i) {
    const Ins& I = P.ins[i];
    const double a = I.op >= APCG_EX_ADD ? r[I.a] : 0.0;
    const double b = I.op >= APCG_EX_ADD && I.op <= APCG_EX_MAX ? r[I.b] : 0.0;
    double v = 0.0;
    switch (I.op) {
      case APCG_EX_SCALAR: v = *P.loads[I.load]; break;
      case APCG_EX_CONST: v = I.c; break;
      case APCG_EX_ADD: v = a + b; break;
      case APCG_EX_SUB: v = a - b; break;
      case APCG_EX_MUL: v = a * b; break;
      case APCG_EX_DIV: v = a / b; break;
      case APCG_EX_MIN: v = fmin(a, b); break;
      case APCG_EX_MAX: v = fmax(a, b); break;
      case APCG_EX_NEG: v = -a; break;
      case APCG_EX_RECIP: v = 1.0 / a; break;
      case APCG_EX_SQRT: v = sqrt(a); break;
      case APCG_EX_ABS: v = fabs(a); break;
      case APCG_EX_SIN: v = sin(a); break;
      case APCG_EX_COS: v = cos(a); break;
      case APCG_EX_EXP: v = exp(a); break;
      case APCG_EX_LOG: v = log(a); break;
    }
    r[i] = v;
  }
  return r[P.n - 1];
}

__global__ void expr_kernel(Prog P, double* out) { *out = eval_prog(P); }

// y += e x, the expression evaluated once per block in the prologue.
__global__ void __launch_bounds__(256) axpy_expr_kernel(Prog P, int64_t n, double* __restrict__ y,
                                                        const double* __restrict__ x) {
  __shared__ double s_a;
  if (threadIdx.x == 0) s_a = eval_prog(P);
  __syncthreads();
  const double a = s_a;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = fma(a, x[i], y[i]);
}

bool is_binary(int op) { return op >= APCG_EX_ADD && op <= APCG_EX_MAX; }
bool is_unary(int op) { return op >= APCG_EX_NEG && op <= APCG_EX_LOG; }
bool exact_op(int op) { return op != APCG_EX_SIN && op != APCG_EX_COS && op != APCG_EX_EXP && op != APCG_EX_LOG; }

const char* op_name(int op) {
  static const char* names[] = {"scalar", "const", "add", "sub", "mul", "div", "min", "max",
                                "neg", "recip", "sqrt", "abs", "sin", "cos", "exp", "log"};
  return op >= 0 && op < (int)(sizeof(names) / sizeof(names[0])) ? names[op] : "?";
}

// Host evaluation of an exactly rounded operation (constant folding).
double host_apply(int op, double a, double b) {
  switch (op) {
    case APCG_EX_ADD: return a + b;
    case APCG_EX_SUB: return a - b;
    case APCG_EX_MUL: return a * b;
    case APCG_EX_DIV: return a / b;
    case APCG_EX_MIN: return std::fmin(a, b);
    case APCG_EX_MAX: return std::fmax(a, b);
    case APCG_EX_NEG: return -a;
    case APCG_EX_RECIP: return 1.0 / a;
    case APCG_EX_SQRT: return std::sqrt(a);
    case APCG_EX_ABS: return std::fabs(a);
  }
  return 0.0;
}

}  // namespace
}  // namespace apcg

struct apcg_expr_s {
  apcg::Prog prog;
  std::vector<apcg_scalar> inputs;  // the distinct input scalars, in load order
  std::string text;                 // the frozen program, one instruction per line
};

namespace apcg {
namespace {

// Builder of the frozen DAG: nodes are hash-consed, so equal subexpressions share one node.
struct Builder {
  std::vector<Ins> nodes;
  std::vector<apcg_scalar> loads;
  std::map<std::tuple<int, int, int, uint64_t>, int> seen;

  int add(Ins I) {
    uint64_t cbits = 0;
    if (I.op == APCG_EX_CONST) memcpy(&cbits, &I.c, sizeof cbits);
    const auto key = std::make_tuple((int)I.op, (int)I.a | ((int)I.load << 8), (int)I.b, cbits);
    auto it = seen.find(key);
    if (it != seen.end()) return it->second;
    nodes.push_back(I);
    const int id = (int)nodes.size() - 1;
    seen[key] = id;
    return id;
  }
  int constant(double c) {
    Ins I{};
    I.op = APCG_EX_CONST;
    I.c = c;
    return add(I);
  }
  bool is_const(int i, double v) const {
    if (nodes[i].op != APCG_EX_CONST) return false;
    const double c = nodes[i].c;
    return c == v && std::signbit(c) == std::signbit(v);
  }
  int unary(int op, int a) {
    if (nodes[a].op == APCG_EX_CONST && exact_op(op)) return constant(host_apply(op, nodes[a].c, 0.0));
    if (op == APCG_EX_NEG && nodes[a].op == APCG_EX_NEG) return nodes[a].a;  // -(-x) = x
    Ins I{};
    I.op = (uint8_t)op;
    I.a = (uint8_t)a;
    return add(I);
  }
  int binary(int op, int a, int b) {
    if (nodes[a].op == APCG_EX_CONST && nodes[b].op == APCG_EX_CONST)
      return constant(host_apply(op, nodes[a].c, nodes[b].c));
    if ((op == APCG_EX_MUL || op == APCG_EX_DIV) && is_const(b, 1.0)) return a;  // x * 1 = x / 1 = x
    if (op == APCG_EX_MUL && is_const(a, 1.0)) return b;
    if (op == APCG_EX_SUB && is_const(b, 0.0)) return a;  // x - (+0) = x, also for x = -0
    Ins I{};
    I.op = (uint8_t)op;
    I.a = (uint8_t)a;
    I.b = (uint8_t)b;
    return add(I);
  }
};

// Keep only the nodes the result depends on, in dependency order.
apcg_status emit(const Builder& B, int root, apcg_expr_s* E) {
  std::vector<int> order, remap(B.nodes.size(), -1);
  std::vector<int> stack{root};
  std::vector<char> state(B.nodes.size(), 0);  // 0 new, 1 open, 2 done
  while (!stack.empty()) {
    const int v = stack.back();
    if (state[v] == 2) {
      stack.pop_back();
      continue;
    }
    const Ins& I = B.nodes[v];
    if (state[v] == 0) {
      state[v] = 1;
      if (is_binary(I.op)) stack.push_back(I.b);
      if (is_binary(I.op) || is_unary(I.op)) stack.push_back(I.a);
      continue;
    }
    state[v] = 2;
    stack.pop_back();
    order.push_back(v);
  }
  APCG_CHECK((int)order.size() <= kMaxIns, "the frozen expression has %d instructions; at most %d are supported",
             (int)order.size(), kMaxIns);
  Prog& P = E->prog;
  P.n = (int32_t)order.size();
  std::vector<int> load_map(B.loads.size(), -1);
  char line[128];
  for (int i = 0; i < P.n; ++i) {
    Ins I = B.nodes[order[i]];
    remap[order[i]] = i;
    if (is_binary(I.op) || is_unary(I.op)) I.a = (uint8_t)remap[I.a];
    if (is_binary(I.op)) I.b = (uint8_t)remap[I.b];
    if (I.op == APCG_EX_SCALAR) {
      if (load_map[I.load] < 0) {
        load_map[I.load] = (int)E->inputs.size();
        E->inputs.push_back(B.loads[I.load]);
      }
      I.load = (uint8_t)load_map[I.load];
      snprintf(line, sizeof line, "r%d = scalar %d\n", i, (int)I.load);
    } else if (I.op == APCG_EX_CONST) {
      snprintf(line, sizeof line, "r%d = const %.17g\n", i, I.c);
    } else if (is_binary(I.op)) {
      snprintf(line, sizeof line, "r%d = %s r%d r%d\n", i, op_name(I.op), (int)I.a, (int)I.b);
    } else {
      snprintf(line, sizeof line, "r%d = %s r%d\n", i, op_name(I.op), (int)I.a);
    }
    E->text += line;
    P.ins[i] = I;
  }
  P.nload = (int32_t)E->inputs.size();
  return APCG_OK;
}

// Resolve the input scalars' device addresses and mark them read on ctx (out is marked by the caller).
void bind_loads(apcg_expr_s* E) {
  for (int j = 0; j < E->prog.nload; ++j) E->prog.loads[j] = E->inputs[j]->dptr;
}

}  // namespace
}  // namespace apcg

using namespace apcg;

extern "C" {

apcg_status apcg_expr_create(const apcg_expr_term* terms, int32_t nterms, apcg_expr* out) {
  APCG_CHECK(terms && out, "NULL argument");
  APCG_CHECK(nterms >= 1 && nterms <= 4 * kMaxIns, "nterms must be in 1..%d", 4 * kMaxIns);
  Builder B;
  std::vector<int> st;
  std::map<apcg_scalar, int> load_index;
  for (int32_t k = 0; k < nterms; ++k) {
    const apcg_expr_term& t = terms[k];
    if (t.op == APCG_EX_SCALAR) {
      APCG_CHECK(t.s, "term %d: NULL scalar", k);
      auto it = load_index.find(t.s);
      int li;
      if (it == load_index.end()) {
        APCG_CHECK((int)B.loads.size() < kMaxLoads, "more than %d distinct input scalars", kMaxLoads);
        li = (int)B.loads.size();
        B.loads.push_back(t.s);
        load_index[t.s] = li;
      } else {
        li = it->second;
      }
      Ins I{};
      I.op = APCG_EX_SCALAR;
      I.load = (uint8_t)li;
      st.push_back(B.add(I));
    } else if (t.op == APCG_EX_CONST) {
      st.push_back(B.constant(t.c));
    } else if (is_binary(t.op)) {
      APCG_CHECK(st.size() >= 2, "term %d (%s): needs two operands", k, op_name(t.op));
      const int b = st.back();
      st.pop_back();
      const int a = st.back();
      st.pop_back();
      st.push_back(B.binary(t.op, a, b));
    } else if (is_unary(t.op)) {
      APCG_CHECK(!st.empty(), "term %d (%s): needs an operand", k, op_name(t.op));
      const int a = st.back();
      st.pop_back();
      st.push_back(B.unary(t.op, a));
    } else {
      return set_error(APCG_ERR_INVALID_ARG, "term %d: unknown operator %d", k, t.op);
    }
    APCG_CHECK(B.nodes.size() <= 255, "expression too large");
  }
  APCG_CHECK(st.size() == 1, "the terms leave %d values instead of one", (int)st.size());
  std::unique_ptr<apcg_expr_s> E(new apcg_expr_s());
  APCG_TRY(emit(B, st.back(), E.get()));
  *out = E.release();
  return APCG_OK;
}

apcg_status apcg_expr_destroy(apcg_expr e) {
  APCG_CHECK(e, "expression is NULL");
  delete e;
  return APCG_OK;
}

apcg_status apcg_expr_describe(apcg_expr e, int32_t* ninstr, int32_t* ninputs, char* text, size_t cap) {
  APCG_CHECK(e, "expression is NULL");
  if (ninstr) *ninstr = e->prog.n;
  if (ninputs) *ninputs = e->prog.nload;
  if (text && cap) {
    const size_t nb = std::min(cap - 1, e->text.size());
    memcpy(text, e->text.data(), nb);
    text[nb] = '\0';
  }
  return APCG_OK;
}

apcg_status apcg_expr_execute_async(apcg_ctx ctx_in, apcg_expr e, apcg_scalar out) {
  APCG_CHECK(e && out, "NULL argument");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  bind_loads(e);
  OpScope op(ctx);
  for (apcg_scalar s : e->inputs) op.read(s->id);
  op.write(out->id);
  APCG_TRY(op.begin());
  expr_kernel<<<1, 1, 0, ctx->stream>>>(e->prog, out->dptr);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_vec_axpy_expr_async(apcg_ctx ctx_in, apcg_vec y, apcg_expr e, apcg_vec x) {
  APCG_CHECK(y && x && e, "NULL argument");
  APCG_CHECK(x->dtype == APCG_F64 && y->dtype == APCG_F64, "x and y must be float64");
  APCG_CHECK(x->n == y->n, "x and y differ in length");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  bind_loads(e);
  OpScope op(ctx);
  for (apcg_scalar s : e->inputs) op.read(s->id);
  op.read(x->id).rw(y->id);
  APCG_TRY(op.begin());
  if (y->n > 0) {
    const int64_t want = (y->n + 255) / 256;
    const int g = (int)std::min<int64_t>(want, (int64_t)8 * ctx_num_sms(ctx));
    axpy_expr_kernel<<<g, 256, 0, ctx->stream>>>(e->prog, y->n, static_cast<double*>(y->dptr),
                                                  static_cast<const double*>(x->dptr));
    APCG_CUDA(cudaGetLastError());
    count_kernels(1);
  }
  return op.finish();
}

}  // extern "C"
