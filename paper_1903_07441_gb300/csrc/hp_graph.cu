// Graph-driven convergence loop for the red-black SOR solve.
//
// One CUDA graph holds a conditional WHILE node whose body is one check
// interval: K/T launches of the T-fused sweep kernel, the FP32 residual
// reduction, a control kernel, a conditional IF node holding the polish (one
// T-sweep launch at omega = 1 into the other ping-pong planes and its
// residual) and a one-thread kernel that takes the polish result and sets the
// loop condition.  The control kernel applies the same decisions as the host
// loop (relax_control: stop at the tolerance, back off over-relaxation at the
// rounding floor, adapt omega; relax_polish_decide), writes the new omega
// where the sweep kernels read it and sets the IF condition.  The host
// launches the graph once per solve and reads the state back once, instead
// of synchronising at every check.  The loop is bounded: the control kernel
// stops after max_intervals intervals.
//
// Instantiated graphs are cached per (device, workspace, grid, T, K): the
// kernel arguments are workspace pointers and shapes, so a cached graph is
// valid for every solve that reuses the same workspace.
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "hp_internal.cuh"

namespace tw {

void tb_kernel_node(int T, RBLayout &L, int ny, void **func, dim3 *grid, dim3 *block);
void *rb_residual_kernel_ptr();

// handle: the loop condition (polish == 0) or the polish IF condition.
// dmax (nullable): the largest change of a free cell over the interval's last launch.
__global__ void relax_control_kernel(RelaxCtl *ctl, unsigned int *rmax, const float *l2part, int n_part,
                                     int max_intervals, cudaGraphConditionalHandle handle, int polish,
                                     unsigned int *dmax) {
    // the 2-norm from the residual kernel's per-CTA partials (whole CTA), then thread 0 decides
    const double e = l2part ? sqrt(block_sum_partials(l2part, n_part, threadIdx.x)) : -1.0;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    RelaxCtl c = *ctl;
    const float rf = __uint_as_float(*rmax);
    *rmax = 0u;
    double d = -1.0;
    if (dmax && c.snap == 2) {   // the residual kernel compared with the snapshot in this interval
        d = (double)__uint_as_float(*dmax);
        *dmax = 0u;
    }
    c.sweeps += c.K;
    const int cont = relax_control(c, (double)rf, e, c.K, d);
    int go = cont;
    if (c.checks >= max_intervals || c.sweeps + c.K > c.max_sweeps) go = 0;
    c.go = go;
    if (polish) {
        relax_polish_decide(c, cont);
        *ctl = c;
        cudaGraphSetConditional(handle, c.polish ? 1u : 0u);
    } else {
        *ctl = c;
        cudaGraphSetConditional(handle, go ? 1u : 0u);
    }
}

// After the (conditional) polish: accept a polished copy that meets the
// tolerance, then set the loop condition.
__global__ void relax_polish_kernel(RelaxCtl *ctl, unsigned int *rmax, cudaGraphConditionalHandle loop_handle) {
    RelaxCtl c = *ctl;
    if (c.polish) {
        const float r2 = __uint_as_float(*rmax);
        *rmax = 0u;
        if (!relax_polish_result(c, (double)r2)) c.go = 0;
        *ctl = c;
    }
    cudaGraphSetConditional(loop_handle, c.go ? 1u : 0u);
}

static cudaError_t add_kernel_node(cudaGraphNode_t *node, cudaGraph_t g, cudaGraphNode_t *prev, void *func,
                                   dim3 grid, dim3 block, void **args) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(node, g, *prev ? prev : nullptr, *prev ? 1 : 0, &kp);
}

// A kernel node that depends on *prev through a programmatic edge: it may be
// scheduled once every CTA of *prev has triggered (griddepcontrol.launch_
// dependents) and waits for *prev's completion itself (griddepcontrol.wait).
static cudaError_t add_kernel_node_pdl(cudaGraphNode_t *node, cudaGraph_t g, cudaGraphNode_t *prev, void *func,
                                       dim3 grid, dim3 block, void **args) {
    cudaGraphNode_t none = nullptr;
    cudaError_t e = add_kernel_node(node, g, &none, func, grid, block, args);
    if (e != cudaSuccess || !*prev) return e;
    cudaGraphEdgeData ed;
    memset(&ed, 0, sizeof(ed));
    ed.type = cudaGraphDependencyTypeProgrammatic;
    ed.from_port = cudaGraphKernelNodePortProgrammatic;
    return cudaGraphAddDependencies(g, prev, node, &ed, 1);
}

struct GraphEntry {
    int dev, nx, ny, T, K, max_intervals, polish, est;
    const void *key;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

static std::mutex g_graph_mutex;
static std::vector<GraphEntry> g_graphs;
constexpr size_t kMaxCachedGraphs = 16;

static int build_graph(RBLayout L, int nx, int ny, int T, int K, int max_intervals, int polish, int est,
                       RelaxScalars *scal, float *l2part, bool pdl, GraphEntry *out) {
    (void)nx;
    cudaGraph_t g = nullptr;
    TW_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    e = cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    // K/T sweep launches alternating the ping-pong planes (an even count, so the
    // planes are back in place when the residual reads them)
    void *func;
    dim3 grid, block;
    tb_kernel_node(T, L, ny, &func, &grid, &block);
    const int n_launch = K / T;
    const float *omega_dev = &scal->ctl.omega_f;
    float omega_unused = 0.0f;
    cudaGraphNode_t prev = nullptr;
    float *R = L.R, *B = L.B, *R2 = L.R2, *B2 = L.B2;
    int ny_ = ny, w4 = L.W4, S = L.S, mw = L.MW;
    const uint32_t *mr = L.MR, *mb = L.MB;
    for (int i = 0; i < n_launch; i++) {
        const float *rin = R, *bin = B;
        float *rout = R2, *bout = B2;
        void *args[] = {(void *)&rin, (void *)&bin, (void *)&rout, (void *)&bout, (void *)&mr, (void *)&mb,
                        (void *)&ny_, (void *)&w4, (void *)&S, (void *)&mw, (void *)&omega_unused,
                        (void *)&omega_dev};
        cudaGraphNode_t node;
        e = pdl ? add_kernel_node_pdl(&node, body, &prev, func, grid, block, args)
                : add_kernel_node(&node, body, &prev, func, grid, block, args);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return TW_ECUDA; }
        prev = node;
        float *t = R; R = R2; R2 = t;
        t = B; B = B2; B2 = t;
    }
    unsigned int *rmax = &scal->max32;
    RelaxCtl *ctl = &scal->ctl;
    const dim3 rgrid = rb_residual_grid(L, ny), rblock(64, 4);
    unsigned int *dmax = est ? &scal->dmax32 : nullptr;
    {   // residual of the current planes (and with an error tolerance the snapshot work)
        RBLayout Lc = L;
        Lc.R = R; Lc.B = B;
        int snap0 = 0;
        const int *snap_dev = est ? &scal->ctl.snap : nullptr;
        void *args[] = {(void *)&Lc, (void *)&ny_, (void *)&rmax, (void *)&l2part, (void *)&snap0,
                        (void *)&snap_dev, (void *)&dmax};
        cudaGraphNode_t node;
        e = add_kernel_node(&node, body, &prev, rb_residual_kernel_ptr(), rgrid, rblock, args);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return TW_ECUDA; }
        prev = node;
    }
    cudaGraphConditionalHandle hp = h;
    if (polish) {
        e = cudaGraphConditionalHandleCreate(&hp, body, 0u, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    }
    {   // control: stop test, omega (and the polish decision)
        const float *part = l2part;
        int n_part = rb_residual_blocks(L, ny);
        int mi = max_intervals, pol = polish;
        void *args[] = {(void *)&ctl, (void *)&rmax, (void *)&part, (void *)&n_part, (void *)&mi, (void *)&hp,
                        (void *)&pol, (void *)&dmax};
        cudaGraphNode_t node;
        e = add_kernel_node(&node, body, &prev, (void *)relax_control_kernel, dim3(1), dim3(kPartThreads), args);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return TW_ECUDA; }
        prev = node;
    }
    if (polish) {   // IF node: T sweeps at omega = 1 from the current planes into the other pair, and their residual
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hp;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        e = cudaGraphAddNode(&inode, body, &prev, nullptr, 1, &ip);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
        cudaGraph_t pbody = ip.conditional.phGraph_out[0];
        const float *rin = R, *bin = B;
        float *rout = R2, *bout = B2;
        const float *one = &scal->ctl.one_f;
        void *args[] = {(void *)&rin, (void *)&bin, (void *)&rout, (void *)&bout, (void *)&mr, (void *)&mb,
                        (void *)&ny_, (void *)&w4, (void *)&S, (void *)&mw, (void *)&omega_unused, (void *)&one};
        cudaGraphNode_t pprev = nullptr, node;
        e = add_kernel_node(&node, pbody, &pprev, func, grid, block, args);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return TW_ECUDA; }
        pprev = node;
        RBLayout Lp = L;
        Lp.R = R2; Lp.B = B2;
        float *no_part = nullptr;
        int no_snap = 0;
        const int *no_snap_dev = nullptr;
        unsigned int *no_dmax = nullptr;
        void *rargs[] = {(void *)&Lp, (void *)&ny_, (void *)&rmax, (void *)&no_part, (void *)&no_snap,
                         (void *)&no_snap_dev, (void *)&no_dmax};
        e = add_kernel_node(&node, pbody, &pprev, rb_residual_kernel_ptr(), rgrid, rblock, rargs);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return TW_ECUDA; }
        prev = inode;
    }
    if (polish) {   // polish result and loop condition
        void *args[] = {(void *)&ctl, (void *)&rmax, (void *)&h};
        cudaGraphNode_t node;
        e = add_kernel_node(&node, body, &prev, (void *)relax_polish_kernel, dim3(1), dim3(1), args);
        if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return TW_ECUDA; }
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    out->graph = g;
    out->exec = exec;
    return TW_OK;
}

int rb_solve_graph(RBLayout &L, int nx, int ny, int T, int K, int max_intervals, int polish, int est,
                   RelaxScalars *scal, float *l2part, cudaStream_t s, int *launches) {
    if (max_intervals < 1) return 1;
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    GraphEntry *ent = nullptr;
    for (auto &g : g_graphs)
        if (g.dev == dev && g.key == (const void *)scal && g.nx == nx && g.ny == ny && g.T == T && g.K == K &&
            g.max_intervals == max_intervals && g.polish == polish && g.est == est)
            ent = &g;
    if (!ent) {
        if (g_graphs.size() >= kMaxCachedGraphs) {
            cudaGraphExecDestroy(g_graphs.front().exec);
            cudaGraphDestroy(g_graphs.front().graph);
            g_graphs.erase(g_graphs.begin());
        }
        GraphEntry ne;
        ne.dev = dev; ne.nx = nx; ne.ny = ny; ne.T = T; ne.K = K; ne.max_intervals = max_intervals;
        ne.polish = polish;
        ne.est = est;
        ne.key = (const void *)scal;
        // sweep launches chained by programmatic edges where the driver takes them, else plain edges
        static bool pdl_ok = true;
        int e = build_graph(L, nx, ny, T, K, max_intervals, polish, est, scal, l2part, pdl_ok, &ne);
        if (e && pdl_ok) {
            pdl_ok = false;
            cudaGetLastError();
            e = build_graph(L, nx, ny, T, K, max_intervals, polish, est, scal, l2part, false, &ne);
        }
        if (e) return e;
        g_graphs.push_back(ne);
        ent = &g_graphs.back();
    }
    TW_CUDA(cudaGraphLaunch(ent->exec, s));
    (void)launches;   // counted by the caller once the number of intervals is known
    return TW_OK;
}

}  // namespace tw
