// Batched single-source BFS over many graphs in one CUDA-graph launch (an
// extension beyond the paper).  The batch graph holds, for each handle, an
// independent chain
//     k_init -> k_batch_root (root read from a device array) -> device-side
//     iteration loop (conditional WHILE node) -> k_batch_output
// so one cudaGraphLaunch runs every BFS, the chains overlapping on the GPU, and
// the same executable graph is replayed with new roots and output pointers.
#include <algorithm>
#include <set>
#include <vector>

#include "ss_device.cuh"

struct slimsell_batch {
  std::vector<slimsell_handle> hs;
  int sr = 0, policy = 0;
  int* d_roots = nullptr;  // [g]
  int** d_dist = nullptr;  // [g] device output pointers (NULL entries allowed)
  int** d_par = nullptr;   // [g]
  ss::Ctl* h_ctl = nullptr;  // [g] pinned copies of the control blocks
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  int pending = 0;
};

namespace ss {

__global__ void k_batch_root(Dev d, const int* roots, int i) { init_root_state(d, roots[i]); }

__global__ void k_batch_output(Dev d, int* const* dist, int* const* par, int i) {
  write_outputs(d, dist[i], par[i]);
}

static ss_status add_kernel(cudaGraph_t g, void* func, dim3 grid, dim3 block, void** args,
                            const cudaGraphNode_t* deps, size_t ndeps, cudaGraphNode_t* out) {
  cudaKernelNodeParams kp = {};
  kp.func = func;
  kp.gridDim = grid;
  kp.blockDim = block;
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  SS_CUDA(cudaGraphAddKernelNode(out, g, deps, ndeps, &kp));
  return SS_OK;
}

static void free_batch(slimsell_batch* b) {
  if (!b) return;
  if (b->done) {
    cudaEventSynchronize(b->done);
    cudaEventDestroy(b->done);
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->d_roots) cudaFree(b->d_roots);
  if (b->d_dist) cudaFree(b->d_dist);
  if (b->d_par) cudaFree(b->d_par);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  delete b;
}

}  // namespace ss

extern "C" {

ss_status slimsell_batch_create(const slimsell_handle* hs, int32_t g, int32_t semiring,
                                int32_t policy, slimsell_batch_handle* out) {
  using namespace ss;
  set_error("");
  if (!out || !hs || g < 1) {
    set_error("slimsell_batch_create: bad arguments");
    return SS_ERR_INVALID;
  }
  *out = nullptr;
  if (semiring < SS_TROPICAL || semiring > SS_SELMAX || policy < SS_V_FULL || policy > SS_V_LEARNED) {
    set_error("slimsell_batch_create: bad semiring or policy");
    return SS_ERR_INVALID;
  }
  std::set<slimsell_handle> seen;
  for (int i = 0; i < g; ++i) {
    if (!hs[i] || !seen.insert(hs[i]).second) {
      set_error("slimsell_batch_create: handle %d is NULL or repeated", i);
      return SS_ERR_INVALID;
    }
  }
  slimsell_batch* b = new slimsell_batch();
  b->hs.assign(hs, hs + g);
  b->sr = semiring;
  b->policy = policy;
  ss_status s = dmalloc(nullptr, (void**)&b->d_roots, sizeof(int) * (size_t)g);
  if (s == SS_OK) s = dmalloc(nullptr, (void**)&b->d_dist, sizeof(int*) * (size_t)g);
  if (s == SS_OK) s = dmalloc(nullptr, (void**)&b->d_par, sizeof(int*) * (size_t)g);
  if (s == SS_OK && cudaHostAlloc((void**)&b->h_ctl, sizeof(Ctl) * (size_t)g, 0) != cudaSuccess)
    s = cuda_fail(cudaGetLastError(), "cudaHostAlloc");
  if (s == SS_OK && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
    s = cuda_fail(cudaGetLastError(), "cudaEventCreate");
  if (s == SS_OK && cudaMemset(b->d_dist, 0, sizeof(int*) * (size_t)g) != cudaSuccess)
    s = cuda_fail(cudaGetLastError(), "cudaMemset");
  if (s == SS_OK && cudaMemset(b->d_par, 0, sizeof(int*) * (size_t)g) != cudaSuccess)
    s = cuda_fail(cudaGetLastError(), "cudaMemset");
  cudaGraph_t graph = nullptr;
  if (s == SS_OK && cudaGraphCreate(&graph, 0) != cudaSuccess)
    s = cuda_fail(cudaGetLastError(), "cudaGraphCreate");
  for (int i = 0; i < g && s == SS_OK; ++i) {
    slimsell_graph* h = b->hs[(size_t)i];
    Dev d = h->dev();
    int idx = i;
    int* roots = b->d_roots;
    int** dist = b->d_dist;
    int** par = b->d_par;
    cudaGraphNode_t n_init, n_root, n_loop, n_out;
    void* a_init[] = {&d};
    s = add_kernel(graph, (void*)k_init, dim3(vertex_grid(h, 256)), dim3(256), a_init, nullptr, 0, &n_init);
    void* a_root[] = {&d, &roots, &idx};
    if (s == SS_OK)
      s = add_kernel(graph, (void*)k_batch_root, dim3(1), dim3(1), a_root, &n_init, 1, &n_root);
    if (s == SS_OK) s = add_loop_node(h, d, semiring, policy, graph, &n_root, 1, &n_loop);
    void* a_out[] = {&d, &dist, &par, &idx};
    if (s == SS_OK)
      s = add_kernel(graph, (void*)k_batch_output, dim3(vertex_grid(h, 256)), dim3(256), a_out,
                     &n_loop, 1, &n_out);
  }
  if (s == SS_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
    b->exec = nullptr;
    s = cuda_fail(cudaGetLastError(), "cudaGraphInstantiate(batch)");
  }
  if (graph) cudaGraphDestroy(graph);
  if (s != SS_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return SS_OK;
}

ss_status slimsell_batch_run(slimsell_batch_handle b, const int32_t* d_roots,
                             int32_t* const* h_dist, int32_t* const* h_parent, void* stream) {
  using namespace ss;
  set_error("");
  if (!b || !d_roots) {
    set_error("slimsell_batch_run: NULL argument");
    return SS_ERR_INVALID;
  }
  const int g = (int)b->hs.size();
  cudaStream_t st = (cudaStream_t)stream;
  for (slimsell_handle hg : b->hs) hg->values_semiring = -1;
  if (b->pending) SS_CUDA(cudaEventSynchronize(b->done));
  std::vector<int> roots((size_t)g);
  SS_CUDA(cudaMemcpyAsync(roots.data(), d_roots, sizeof(int) * (size_t)g, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < g; ++i)
    if (roots[(size_t)i] < 0 || roots[(size_t)i] >= b->hs[(size_t)i]->n) {
      set_error("slimsell_batch_run: root %d of graph %d out of range", roots[(size_t)i], i);
      return SS_ERR_INVALID;
    }
  std::vector<int*> dist((size_t)g, nullptr), par((size_t)g, nullptr);
  for (int i = 0; i < g; ++i) {
    if (h_dist) dist[(size_t)i] = h_dist[i];
    if (h_parent) par[(size_t)i] = h_parent[i];
  }
  SS_CUDA(cudaMemcpyAsync(b->d_roots, d_roots, sizeof(int) * (size_t)g, cudaMemcpyDeviceToDevice, st));
  SS_CUDA(cudaMemcpyAsync(b->d_dist, dist.data(), sizeof(int*) * (size_t)g, cudaMemcpyHostToDevice, st));
  SS_CUDA(cudaMemcpyAsync(b->d_par, par.data(), sizeof(int*) * (size_t)g, cudaMemcpyHostToDevice, st));
  for (auto* h : b->hs) {
    if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));
    h->pending = 0;
  }
  SS_CUDA(cudaGraphLaunch(b->exec, st));
  for (int i = 0; i < g; ++i)
    SS_CUDA(cudaMemcpyAsync(b->h_ctl + i, b->hs[(size_t)i]->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaEventRecord(b->done, st));
  b->pending = 1;
  return SS_OK;
}

ss_status slimsell_batch_get_stats(slimsell_batch_handle b, ss_run_stats* out) {
  using namespace ss;
  if (!b || !out) {
    set_error("slimsell_batch_get_stats: NULL argument");
    return SS_ERR_INVALID;
  }
  if (b->pending) SS_CUDA(cudaEventSynchronize(b->done));
  b->pending = 0;
  int err = 0;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    const Ctl& c = b->h_ctl[i];
    ss_run_stats r = {};
    r.iterations = c.k - 1;
    r.semiring = b->sr;
    r.reached = (long long)c.reached;
    r.reached_degree = (long long)c.reached_deg;
    r.slots = (long long)c.total_slots;
    out[i] = r;
    err |= c.error;
  }
  if (err) {
    set_error("slimsell_batch: iteration limit reached (device error flags %d)", err);
    return SS_ERR_CUDA;
  }
  return SS_OK;
}

void slimsell_batch_destroy(slimsell_batch_handle b) { ss::free_batch(b); }

}  // extern "C"
