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

__device__ __forceinline__ double band_energy(const float *u, int nx, int qx, int qy, const int *path, int i,
                                              double w, double k) {
    double uq = (double)u[(size_t)qy * nx + qx];
    double ax = qx - path[2 * (i - 1)], ay = qy - path[2 * (i - 1) + 1];
    double bx = qx - path[2 * (i + 1)], by = qy - path[2 * (i + 1) + 1];
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
                double best = band_energy(u, nx, px, py, path, i, w, k);
                int nxp = px, nyp = py;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        if (dx == 0 && dy == 0) continue;
                        int qx = px + dx, qy = py + dy;
                        if (qx < 0 || qy < 0 || qx >= nx || qy >= ny) continue;
                        size_t c = (size_t)qy * nx + qx;
                        if (occ[c] != 0) continue;
                        if (!(u[c] > 0.0f)) continue;
                        if (abs(qx - ax) > 1 || abs(qy - ay) > 1 || abs(qx - bx_) > 1 || abs(qy - by_) > 1) continue;
                        double e = band_energy(u, nx, qx, qy, path, i, w, k);
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
