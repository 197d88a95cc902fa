// Path extraction (Eq. 3) and rubber-band smoothing (Sec. 3.2, Eqs. 4-6).
//
// descent_kernel: one CTA.  The walk is inherently serial, so the CTA loads a
// 48x48 window of u around the walker into shared memory in one coalesced
// pass and a single thread takes as many steps as stay inside the window
// before the next reload: one global round trip per ~20 steps instead of one
// per step.
// band_kernel: one CTA.  A rubber-band sweep moves all odd interior nodes in
// parallel, then all even ones (nodes of one parity only read nodes of the
// other parity), so it is exactly the sequential odd-then-even sweep.
#include <math.h>

#include "common.cuh"

namespace tw {

constexpr int kWin = 48;
constexpr int kPathThreads = 512;

struct PathOut {
    int len;
    int status;
    int sweeps;
    int pad;
};

__global__ void __launch_bounds__(kPathThreads)
descent_kernel(const float *__restrict__ u, const uint8_t *__restrict__ occ, int nx, int ny, int sx, int sy,
               int gx, int gy, int max_len, int *__restrict__ path, PathOut *out) {
    __shared__ float win[kWin][kWin];
    __shared__ int s_x, s_y, s_len, s_status, s_done;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_x = sx; s_y = sy; s_len = 1; s_status = TW_OK; s_done = 0;
        bool at_goal = (sx == gx && sy == gy);
        if (occ[(size_t)sy * nx + sx] != 0 && !at_goal) { s_status = TW_ESTART_BLOCKED; s_done = 1; s_len = 0; }
        else { path[0] = sx; path[1] = sy; }
    }
    __syncthreads();
    while (!s_done) {
        const int wx0 = s_x - kWin / 2, wy0 = s_y - kWin / 2;
        for (int idx = tid; idx < kWin * kWin; idx += kPathThreads) {
            int i = idx % kWin, j = idx / kWin;
            int x = wx0 + i, y = wy0 + j;
            win[j][i] = (x >= 0 && y >= 0 && x < nx && y < ny) ? u[(size_t)y * nx + x] : -INFINITY;
        }
        __syncthreads();
        if (tid == 0) {
            int x = s_x, y = s_y, L = s_len;
            const int DX[4] = {1, -1, 0, 0}, DY[4] = {0, 0, 1, -1};
            for (;;) {
                if (x == gx && y == gy) { s_done = 1; s_status = TW_OK; break; }
                int lx = x - wx0, ly = y - wy0;
                if (lx < 1 || ly < 1 || lx > kWin - 2 || ly > kWin - 2) break;  // reload the window
                float bu = win[ly][lx];
                int best = -1;
                for (int k = 0; k < 4; k++) {
                    float v = win[ly + DY[k]][lx + DX[k]];
                    if (v > bu) { bu = v; best = k; }
                }
                if (best < 0 || L >= max_len) { s_done = 1; s_status = TW_NO_PATH; break; }
                x += DX[best]; y += DY[best];
                path[2 * L] = x; path[2 * L + 1] = y;
                L++;
            }
            s_x = x; s_y = y; s_len = L;
        }
        __syncthreads();
    }
    if (tid == 0) { out->len = s_len; out->status = s_status; }
}

// Energy of node position q between its neighbours a and b (u_q = u at q).
__device__ __forceinline__ double band_energy_q(float u_q, int qx, int qy, int pax, int pay, int pbx, int pby,
                                                double w, double k) {
    double uq = (double)u_q;
    double ax = qx - pax, ay = qy - pay;
    double bx = qx - pbx, by = qy - pby;
    return __dadd_rn(__ddiv_rn(w, uq),
                     __dmul_rn(__dmul_rn(0.5, k),
                               __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)),
                                         __dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)))));
}

__global__ void __launch_bounds__(kPathThreads)
band_kernel(const float *__restrict__ u, const uint8_t *__restrict__ occ, int nx, int ny, int *path, PathOut *out,
            int iters, double w, double k) {
    __shared__ int s_moved;
    const int L = out->len;
    if (out->status != TW_OK || L < 3) {
        if (threadIdx.x == 0) out->sweeps = 0;
        return;
    }
    int s = 0;
    for (; s < iters; s++) {
        if (threadIdx.x == 0) s_moved = 0;
        __syncthreads();
        for (int parity = 1; parity >= 0; parity--) {
            for (int i = 2 * threadIdx.x + parity; i < L - 1; i += 2 * kPathThreads) {
                if (i < 1) continue;
                int px = path[2 * i], py = path[2 * i + 1];
                int ax = path[2 * (i - 1)], ay = path[2 * (i - 1) + 1];
                int bx_ = path[2 * (i + 1)], by_ = path[2 * (i + 1) + 1];
                // the 3 x 3 neighbourhood's u and occupancy, loaded together (one round trip
                // instead of one per candidate); outside the grid reads as occupied
                float uq[9];
                uint8_t oq[9];
#pragma unroll
                for (int t = 0; t < 9; t++) {
                    const int qx = px + t % 3 - 1, qy = py + t / 3 - 1;
                    const bool in = qx >= 0 && qy >= 0 && qx < nx && qy < ny;
                    const size_t c = in ? (size_t)qy * nx + qx : 0;
                    uq[t] = in ? u[c] : 0.0f;
                    oq[t] = in ? occ[c] : (uint8_t)1;
                }
                // FP32 screen: a candidate whose FP32 energy exceeds the smallest by more than a
                // relative 1e-5 cannot be the FP64 minimum (the FP32 values carry a relative error
                // below 1e-6 and every energy is positive), so only the near-minimal candidates
                // take the FP64 energies the decision is made with
                float e32[9];   // NaN: not a candidate; +inf (FP32 overflow): always checked in FP64
                float m32 = INFINITY;
                const float w32 = (float)w, hk32 = 0.5f * (float)k;
#pragma unroll
                for (int t = 0; t < 9; t++) {
                    e32[t] = __int_as_float(0x7fc00000);
                    if (t == 4) continue;
                    const int qx = px + t % 3 - 1, qy = py + t / 3 - 1;
                    if (oq[t] != 0) continue;
                    if (!(uq[t] > 0.0f)) continue;
                    if (abs(qx - ax) > 1 || abs(qy - ay) > 1 || abs(qx - bx_) > 1 || abs(qy - by_) > 1) continue;
                    const int d2 = (qx - ax) * (qx - ax) + (qy - ay) * (qy - ay) + (qx - bx_) * (qx - bx_) +
                                   (qy - by_) * (qy - by_);
                    e32[t] = w32 / uq[t] + hk32 * (float)d2;
                    m32 = fminf(m32, e32[t]);
                }
                double best = band_energy_q(uq[4], px, py, ax, ay, bx_, by_, w, k);
                int nxp = px, nyp = py;
                const float lim = m32 * (1.0f + 1e-5f);
#pragma unroll
                for (int t = 0; t < 9; t++) {   // dy outer, dx inner, as listed
                    if (t == 4 || e32[t] != e32[t] || (e32[t] > lim && e32[t] != INFINITY)) continue;
                    const int qx = px + t % 3 - 1, qy = py + t / 3 - 1;
                    double e = band_energy_q(uq[t], qx, qy, ax, ay, bx_, by_, w, k);
                    if (e < best) { best = e; nxp = qx; nyp = qy; }
                }
                if (nxp != px || nyp != py) {
                    path[2 * i] = nxp; path[2 * i + 1] = nyp;
                    s_moved = 1;
                }
            }
            __syncthreads();
        }
        int moved = s_moved;
        __syncthreads();
        if (!moved) { s++; break; }
    }
    if (threadIdx.x == 0) {
        int o = 1;
        for (int i = 1; i < L; i++) {
            if (path[2 * i] == path[2 * (o - 1)] && path[2 * i + 1] == path[2 * (o - 1) + 1]) continue;
            path[2 * o] = path[2 * i]; path[2 * o + 1] = path[2 * i + 1];
            o++;
        }
        out->len = o;
        out->sweeps = s;
    }
}

static size_t carve_path(Carver &cv, int max_len, int **path, PathOut **out) {
    PathOut *o = cv.take<PathOut>(1);
    int *p = cv.take<int>((size_t)2 * (max_len > 0 ? max_len : 1));
    if (path) *path = p;
    if (out) *out = o;
    return cv.need;
}

}  // namespace tw

using namespace tw;

extern "C" size_t plan_path_workspace_size(int max_len) {
    Carver cv;
    return carve_path(cv, max_len, nullptr, nullptr);
}

extern "C" int plan_path_ex(const tw_grid *g, const float *u_dev, const uint8_t *occ_dev, int sx, int sy,
                            int gx, int gy, int rubber_iters, double w, double k, int max_len,
                            int32_t *path_xy_host, int *len_out, void *workspace, size_t workspace_bytes,
                            void *stream) {
    if (!g || g->nx < 3 || g->ny < 3 || !u_dev || !occ_dev || !path_xy_host || !len_out || max_len < 1 ||
        rubber_iters < 0 || !isfinite(w) || !isfinite(k) || w < 0.0 || k < 0.0)
        return TW_EINVAL;
    *len_out = 0;
    int nx = g->nx, ny = g->ny;
    if (sx < 0 || sy < 0 || sx >= nx || sy >= ny || gx < 0 || gy < 0 || gx >= nx || gy >= ny) return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace)) return TW_EWORKSPACE;
    Carver cv(workspace, workspace_bytes);
    int *path = nullptr;
    PathOut *out = nullptr;
    carve_path(cv, max_len, &path, &out);
    if (!cv.ok()) return TW_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    TW_LAUNCH(descent_kernel, 1, kPathThreads, 0, s, u_dev, occ_dev, nx, ny, sx, sy, gx, gy, max_len, path, out);
    TW_CHECK_LAUNCH();
    TW_LAUNCH(band_kernel, 1, kPathThreads, 0, s, u_dev, occ_dev, nx, ny, path, out, rubber_iters, w, k);
    TW_CHECK_LAUNCH();
    PathOut h;
    TW_CUDA(cudaMemcpyAsync(&h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaStreamSynchronize(s));
    if (h.len > 0) {
        TW_CUDA(cudaMemcpyAsync(path_xy_host, path, sizeof(int) * 2 * (size_t)h.len, cudaMemcpyDeviceToHost, s));
        TW_CUDA(cudaStreamSynchronize(s));
    }
    *len_out = h.len;
    return h.status;
}

extern "C" int plan_path(const tw_grid *g, const float *u_dev, const uint8_t *occ_dev, int sx, int sy, int gx,
                         int gy, int rubber_iters, int max_len, int32_t *path_xy_host, int *len_out,
                         void *workspace, size_t workspace_bytes, void *stream) {
    return plan_path_ex(g, u_dev, occ_dev, sx, sy, gx, gy, rubber_iters, 1e-3, 1.0, max_len, path_xy_host,
                        len_out, workspace, workspace_bytes, stream);
}
