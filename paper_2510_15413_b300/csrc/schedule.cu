// schedule.cu -- the circuit scheduler's device half: a scan's gate
// descriptors generated on the GPU from its per-row netlist (Alg. 2 runs
// EvaluateHomomorphicTree on every row; here the rows' gates are laid out
// level by level, gate-major within a level, rows in order: descriptor
// (level L, j-th gate of the level, row r) is at level_offset[L] + j rows + r).
//
// A scan program is the per-row netlist (gate types, input wire ids, the
// level order of the gates, the scratch slot of every intermediate wire)
// plus the scan's buffer pointers, a few kilobytes in all; one kernel then
// writes rows x gates descriptors (40 B each) straight into device memory,
// so a plan upload or a served query's admission copies the program instead
// of hundreds of megabytes of host-built descriptors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "engine.h"

namespace fsql {
namespace {

constexpr int kProgMaxPayloads = 64;

// Header of a scan program in device memory, followed by int32 arrays of
// `gates` entries each: order (gate ids in level order), type, a, b, c
// (-1: no third input), slot (scratch slot of the gate's output, -1 for the
// match gate and the mask gates).
struct ProgHeader {
  uint64_t rows;
  uint64_t words;
  int32_t width, n_const, n_inputs, first_mask, match_wire, payload_width, gates, n_int;
  const uint32_t* column;
  const uint32_t* cst;
  uint32_t* match;
  uint32_t* wires;
  const uint32_t* payloads[kProgMaxPayloads];
  uint32_t* outs[kProgMaxPayloads];
};

__device__ __forceinline__ uint32_t* gate_out_ptr(const ProgHeader& h, const int32_t* slot, int g, size_t row) {
  const size_t W = h.words;
  if (g >= h.first_mask) {
    const int m = g - h.first_mask;
    return h.outs[m / h.payload_width] + (row * h.payload_width + m % h.payload_width) * W;
  }
  if (h.n_inputs + g == h.match_wire) return h.match + row * W;
  return h.wires + (row * static_cast<size_t>(h.n_int) + slot[g]) * W;
}

__device__ __forceinline__ const uint32_t* wire_ptr(const ProgHeader& h, const int32_t* slot, int id, size_t row) {
  const size_t W = h.words;
  if (id < h.width) return h.column + (row * h.width + id) * W;
  if (id < h.width + h.n_const) return h.cst + static_cast<size_t>(id - h.width) * W;
  if (id < h.n_inputs) {
    const int m = id - h.width - h.n_const;
    return h.payloads[m / h.payload_width] + (row * h.payload_width + m % h.payload_width) * W;
  }
  return gate_out_ptr(h, slot, id - h.n_inputs, row);
}

// Descriptor d of the scan: gate order[d / rows] of row d % rows.
__global__ void gen_desc_kernel(const ProgHeader* __restrict__ prog, GateDesc* __restrict__ out, size_t total) {
  __shared__ ProgHeader h;
  for (int k = threadIdx.x; k < static_cast<int>(sizeof(ProgHeader) / 8); k += blockDim.x)
    reinterpret_cast<uint64_t*>(&h)[k] = reinterpret_cast<const uint64_t*>(prog)[k];
  __syncthreads();
  const int32_t* arr = reinterpret_cast<const int32_t*>(prog + 1);
  const int G = h.gates;
  const int32_t *order = arr, *type = arr + G, *a = arr + 2 * G, *b = arr + 3 * G, *c = arr + 4 * G,
                *slot = arr + 5 * G;
  for (size_t d = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; d < total;
       d += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t row = d % h.rows;
    const int g = __ldg(order + d / h.rows);
    GateDesc o;
    o.a = wire_ptr(h, slot, __ldg(a + g), row);
    o.b = wire_ptr(h, slot, __ldg(b + g), row);
    const int cg = __ldg(c + g);
    o.c = cg >= 0 ? wire_ptr(h, slot, cg, row) : nullptr;
    o.out = gate_out_ptr(h, slot, g, row);
    o.type = static_cast<uint32_t>(__ldg(type + g));
    o.pad = 0;
    out[d] = o;
  }
}

}  // namespace

size_t scan_program_bytes(const Netlist& nl) { return sizeof(ProgHeader) + 6 * nl.type.size() * sizeof(int32_t); }

bool build_scan_program(const Netlist& nl, const ScanIO& io, std::vector<uint8_t>* out,
                        std::vector<size_t>* level_offset) {
  if (io.n_payloads > static_cast<uint32_t>(kProgMaxPayloads)) return false;
  const int G = static_cast<int>(nl.type.size());
  out->assign(scan_program_bytes(nl), 0);
  ProgHeader h;
  std::memset(&h, 0, sizeof(h));
  h.rows = io.rows;
  h.words = io.words;
  h.width = static_cast<int32_t>(io.width);
  h.n_const = nl.n_const;
  h.n_inputs = nl.n_inputs;
  h.first_mask = nl.first_mask_gate;
  h.match_wire = nl.match_wire;
  h.payload_width = static_cast<int32_t>(std::max<uint32_t>(io.payload_width, 1));
  h.gates = G;
  h.n_int = static_cast<int32_t>(scan_internal_wires(nl));
  h.column = io.column;
  h.cst = io.cst;
  h.match = io.match;
  h.wires = io.wires;
  for (uint32_t q = 0; q < io.n_payloads; ++q) {
    h.payloads[q] = io.payloads[q];
    h.outs[q] = io.outs[q];
  }
  std::memcpy(out->data(), &h, sizeof(h));
  int32_t* arr = reinterpret_cast<int32_t*>(out->data() + sizeof(ProgHeader));
  // gates in level order (stable: netlist order within a level)
  std::vector<int32_t> order(G);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nl.level[x] < nl.level[y]; });
  int32_t n_int = 0;
  for (int g = 0; g < G; ++g) {
    arr[g] = order[g];
    arr[G + g] = nl.type[g];
    arr[2 * G + g] = nl.a[g];
    arr[3 * G + g] = nl.b[g];
    arr[4 * G + g] = nl.c[g];
    arr[5 * G + g] = (g < nl.first_mask_gate && nl.n_inputs + g != nl.match_wire) ? n_int++ : -1;
  }
  level_offset->assign(nl.levels + 1, 0);
  std::vector<size_t> per_level(nl.levels + 1, 0);
  for (int g = 0; g < G; ++g) ++per_level[nl.level[g]];
  size_t pos = 0;
  for (int L = 1; L <= nl.levels; ++L) {
    (*level_offset)[L - 1] = pos;
    pos += per_level[L] * io.rows;
  }
  (*level_offset)[nl.levels] = pos;
  return true;
}

int launch_gen_desc(const void* d_prog, GateDesc* d_out, size_t total, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (total == 0) return FSQL_OK;
  const unsigned blocks = static_cast<unsigned>(std::min<size_t>((total + 255) / 256, 4096));
  gen_desc_kernel<<<blocks, 256, 0, st>>>(static_cast<const ProgHeader*>(d_prog), d_out, total);
  return cudaGetLastError() == cudaSuccess ? FSQL_OK : FSQL_ERR_CUDA;
}

}  // namespace fsql
