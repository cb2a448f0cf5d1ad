// Host check of the low-diagonal tables built by solver.cu (no GPU needed):
//  1. every shared-memory index that any table entry of any class can produce
//     lies inside that class's planes;
//  2. each class's resolved program, run on the compact planes through the
//     kernel's own per-node functions (their host builds), gives bit for bit
//     the values of a plain recursive W-cycle of Algorithm 1 (with the same
//     two program simplifications: the restriction clears the child's
//     correction, and diagonal 0 is solved once per diagonal-1 visit) run on
//     full node arrays of every grid.
// Built and run by tests/test_low_tables.py.
#include "../paper_1907_12334_gb300/csrc/solver.cu"
#include <cstring>
#include <functional>
#include <random>
using namespace msg;
typedef float T;
struct Grid { int p, q, nx, ny, W; std::vector<T> U, B, AX, AY; };

static int check_bounds()
{
    const LowTables& lt = low_tables();
    int bad = 0;
    for (int dl = 0; dl <= kDW; ++dl)
        for (int pic = 1; pic <= dl + 1; ++pic)
            for (int qic = 1; qic <= dl + 1; ++qic) {
                const LowDesc& D = lt.desc[low_class(pic, qic, dl)];
                if (D.nu + D.nb + D.nfx + D.nfy > kLowSlot) { printf("slot\n"); bad++; }
                auto in = [&](long v, long n, const char* w) { if (v < 0 || v >= n) { if (bad < 20) printf("OOB %s %ld/%ld cls %d %d %d\n", w, v, n, pic, qic, dl); bad++; } };
                auto node = [&](int c, int bi, int xf, int yf, int W) {
                    in(c, D.nu, "u"); in(c - 1, D.nu, "u"); in(c + 1, D.nu, "u"); in(c - W, D.nu, "u"); in(c + W, D.nu, "u");
                    in(bi, D.nb, "b"); in(xf - 1, D.nfx, "fx"); in(xf, D.nfx, "fx"); in(yf, D.nfy, "fy"); in(yf + W - 2, D.nfy, "fy");
                };
                for (int d = 0; d <= dl; ++d) {
                    for (int k = 0; k < 2; ++k)
                        for (int e = 0; e < D.cnt[d][k]; ++e) {
                            uint2 v = lt.ent[D.off[d][k] + e];
                            node(v.x & 0x3FF, (v.x >> 10) & 0x3FF, v.y & 0xFFFF, v.y >> 16, v.x >> 20);
                        }
                    for (int e = 0; e < D.cnt[d][LK_RESTRICT]; ++e) {
                        uint2 a = lt.ent[D.off[d][LK_RESTRICT] + 2 * e], f = lt.ent[D.off[d][LK_RESTRICT] + 2 * e + 1];
                        int cu = a.x & 0x3FF, cb = (a.x >> 10) & 0x3FF, Wc = (a.x >> 20) & 0x3F; bool hx = (a.x >> 26) & 1, hy = (a.x >> 27) & 1;
                        in(cu, D.nu, "cu"); in(cb, D.nb, "cb");
                        if (!hx && !hy) { printf("no parent\n"); bad++; }
                        if (hx) { int pu = a.y & 0x3FF, pb = (a.y >> 10) & 0x3FF, px = a.y >> 20, py = f.x & 0x3FF, W = 2 * Wc - 1;
                                  for (int s = -1; s <= 1; ++s) node(pu + s, pb + s, px + s, py + s, W); }
                        if (hy) { int qu = (f.x >> 10) & 0x3FF, qb = f.x >> 20, qx = f.y & 0x3FF, qy = f.y >> 10, W = Wc;
                                  for (int s = -1; s <= 1; ++s) node(qu + s * W, qb + s * (W - 2), qx + s * (W - 1), qy + s * (W - 2), W); }
                    }
                    for (int e = 0; e < D.cnt[d][LK_PROL]; ++e) {
                        uint2 v = lt.ent[D.off[d][LK_PROL] + e];
                        int c = v.x & 0x3FF, W = (v.x >> 10) & 0x3F, xf = v.x >> 20; bool io = (v.x >> 16) & 1, jo = (v.x >> 17) & 1, hx = (v.x >> 18) & 1, hy = (v.x >> 19) & 1;
                        int rx = v.y & 0x3FF, ry = (v.y >> 10) & 0x3FF, yf = v.y >> 20;
                        in(c, D.nu, "pc"); in(xf - 1, D.nfx, "pfx"); in(xf, D.nfx, "pfx"); in(yf, D.nfy, "pfy"); in(yf + W - 2, D.nfy, "pfy");
                        if (hx) { in(rx, D.nu, "rx"); if (io) in(rx + 1, D.nu, "rx1"); }
                        if (hy) { in(ry, D.nu, "ry"); if (jo) in(ry + W, D.nu, "ryW"); }
                    }
                }
                for (int g = 0; g < D.ngrid; ++g) {
                    int w = D.grid[g], p = w & 15, q = (w >> 4) & 15, nx = 1 << p, ny = 1 << q;
                    in((w >> 8) + low_nodes(p, q) - 1, D.nu, "grid u"); in(D.gb[g] + (nx - 1) * (ny - 1) - 1, D.nb, "grid b");
                    in(D.gx[g] + nx * (ny - 1) - 1, D.nfx, "grid fx"); in(D.gy[g] + (nx - 1) * ny - 1, D.nfy, "grid fy");
                }
            }
    for (int mu = 1; mu <= 3; ++mu)
        for (int nu = 0; nu <= 3; ++nu) {
            msg_params prm{}; prm.mu = mu; prm.nu1 = nu; prm.nu2 = nu ? nu : 1;
            std::vector<LowDesc> desc;
            std::vector<uint2> rp = low_resolve(prm, desc);
            for (const LowDesc& D : desc)
                for (int o = 0; o < D.nops; ++o) {
                    uint2 w = rp[D.prog + o]; int kind = w.x & 7, cnt = w.x >> 3, off = w.y;
                    size_t words = (size_t)cnt * (kind == LK_RESTRICT ? 2 : 1);
                    if (kind >= LK_NKIND || cnt <= 0 || off < 0 || off + words > lt.ent.size()) bad++;
                }
        }
    printf("bounds: slot %d values, %zu table words, %d out of range\n", kLowSlot, lt.ent.size(), bad);
    return bad;
}

static int check_program()
{
    const LowTables& lt = low_tables();
    std::mt19937 rng(1);
    std::uniform_real_distribution<float> ud(0.05f, 3.0f), ub(-1.f, 1.f);
    int bad = 0, checked = 0;
    for (int mu = 1; mu <= 3; ++mu)
    for (int nu = 1; nu <= 2; ++nu)
    for (int dl = 0; dl <= kDW; ++dl)
    for (int pic = 1; pic <= dl + 1; ++pic)
    for (int qic = 1; qic <= dl + 1; ++qic) {
        if (pic + qic < dl + 2) continue;  // no item has such a class
        msg_params prm{}; prm.mu = mu; prm.nu1 = nu; prm.nu2 = nu; prm.omega = 1.0;
        std::vector<LowDesc> desc;
        std::vector<uint2> rp = low_resolve(prm, desc);
        const LowDesc& D = desc[low_class(pic, qic, dl)];
        auto exists = [&](int p, int q) { return p >= 1 && q >= 1 && p <= pic && q <= qic && p + q - 2 <= dl; };
        Grid G[8][8];
        for (int p = 1; p <= 6; ++p) for (int q = 1; q <= 6; ++q) if (exists(p, q)) {
            Grid& g = G[p][q]; g.p = p; g.q = q; g.nx = 1 << p; g.ny = 1 << q; g.W = g.nx + 1;
            int n = (g.nx + 1) * (g.ny + 1);
            g.U.assign(n, 0.f); g.B.assign(n, 0.f); g.AX.resize(n); g.AY.resize(n);
            for (auto& v : g.AX) v = ud(rng);
            for (auto& v : g.AY) v = ud(rng);
            if (p + q - 2 == dl) for (int j = 1; j < g.ny; ++j) for (int i = 1; i < g.nx; ++i) g.B[j * g.W + i] = ub(rng);
        }
        // ---- compact planes filled like the kernel's prologue
        std::vector<T> plane(kLowSlot, -777.f);
        T* u = plane.data(); T* b = u + D.nu; T* fx = b + D.nb; T* fy = fx + D.nfx;
        if (D.nu + D.nb + D.nfx + D.nfy > kLowSlot) { printf("slot overflow\n"); bad++; }
        for (int k = 0; k < D.nu; ++k) u[k] = 0;
        for (int g = 0; g < D.ngrid; ++g) {
            int w = D.grid[g], p = w & 15, q = (w >> 4) & 15, nx = 1 << p, W = nx + 1;
            Grid& gr = G[p][q];
            for (int k = 0; k < (((1 << q) - 1) << p); ++k) { int i = k & (nx - 1), j = 1 + (k >> p); fx[D.gx[g] + k] = gr.AX[j * W + i]; }
            for (int k = 0; k < ((1 << q) << p); ++k) { int i = k & (nx - 1), j = k >> p; if (!i) continue; fy[D.gy[g] + j * (nx - 1) + i - 1] = gr.AY[j * W + i]; }
            if (p + q - 2 == dl)
                for (int k = 0; k < (((1 << q) - 1) << p); ++k) { int i = k & (nx - 1), j = 1 + (k >> p); if (!i) continue; b[D.gb[g] + (j - 1) * (nx - 1) + i - 1] = gr.B[j * W + i]; }
        }
        // ---- the program, twice (two mu-cycles, as the kernel's calls = 2)
        for (int call = 0; call < 2; ++call)
            for (int o = 0; o < D.nops; ++o) {
                uint2 op = rp[D.prog + o]; int kind = op.x & 7, cnt = op.x >> 3, off = op.y;
                for (int k = 0; k < cnt; ++k) {
                    if (kind <= LK_SMOOTH_BLACK) low_smooth(u, b, fx, fy, lt.ent[off + k]);
                    else if (kind == LK_RESTRICT) low_restrict(u, b, fx, fy, lt.ent[off + 2 * k], lt.ent[off + 2 * k + 1]);
                    else low_prol(u, fx, fy, lt.ent[off + k], (T)1.0);
                }
            }
        // ---- reference: plain recursion on full node arrays
        auto res = [&](Grid& g, int i, int j) {
            int c = j * g.W + i, W = g.W;
            T aw = g.AX[c - 1], ae = g.AX[c], as = g.AY[c - W], an = g.AY[c];
            T Au = (aw + ae + as + an) * g.U[c] - (aw * g.U[c - 1] + ae * g.U[c + 1]) - (as * g.U[c - W] + an * g.U[c + W]);
            return g.B[c] - Au;
        };
        auto smooth = [&](int d, int colour) {
            for (int p = 1; p <= d + 1; ++p) { int q = d + 2 - p; if (!exists(p, q)) continue; Grid& g = G[p][q]; int W = g.W;
                for (int j = 1; j < g.ny; ++j) for (int i = 1; i < g.nx; ++i) if (((i + j) & 1) == colour) {
                    int c = j * W + i; T aw = g.AX[c - 1], ae = g.AX[c], as = g.AY[c - W], an = g.AY[c];
                    T nb = (aw * g.U[c - 1] + ae * g.U[c + 1]) + (as * g.U[c - W] + an * g.U[c + W]);
                    g.U[c] = (g.B[c] + nb) * (1.0f / (aw + ae + as + an)); } }
        };
        auto restrict_ = [&](int d) {
            for (int p = 1; p <= d; ++p) { int q = d + 1 - p; if (!exists(p, q)) continue;
                bool hx = exists(p + 1, q), hy = exists(p, q + 1); if (!hx && !hy) continue; Grid& c = G[p][q];
                for (int j = 1; j < c.ny; ++j) for (int i = 1; i < c.nx; ++i) {
                    T vx = 0, vy = 0;
                    if (hx) { Grid& g = G[p + 1][q]; vx = T(0.25) * (res(g, 2 * i - 1, j) + T(2) * res(g, 2 * i, j) + res(g, 2 * i + 1, j)); }
                    if (hy) { Grid& g = G[p][q + 1]; vy = T(0.25) * (res(g, i, 2 * j - 1) + T(2) * res(g, i, 2 * j) + res(g, i, 2 * j + 1)); }
                    c.B[j * c.W + i] = (hx && hy) ? T(0.5) * vx + T(0.5) * vy : (hx ? vx : vy);
                    c.U[j * c.W + i] = 0; } }
        };
        auto prolong = [&](int d) {
            for (int p = 1; p <= d + 1; ++p) { int q = d + 2 - p; if (!exists(p, q)) continue; Grid& g = G[p][q]; int W = g.W;
                bool hx = p > 1, hy = q > 1;
                for (int j = 1; j < g.ny; ++j) for (int i = 1; i < g.nx; ++i) {
                    int c = j * W + i; T vx = 0, vy = 0;
                    if (hx) { Grid& k = G[p - 1][q]; int r = j * k.W + (i >> 1); vx = (i & 1) ? T(0.5) * (k.U[r] + k.U[r + 1]) : k.U[r]; }
                    if (hy) { Grid& k = G[p][q - 1]; int r = (j >> 1) * W + i; vy = (j & 1) ? T(0.5) * (k.U[r] + k.U[r + W]) : k.U[r]; }
                    T corr;
                    if (hx && hy) { T cxv = g.AX[c - 1] + g.AX[c], cyv = g.AY[c - W] + g.AY[c]; T x2 = cxv * cxv, y2 = cyv * cyv, s = 1.0f / (x2 + y2); corr = (x2 * s) * vx + (y2 * s) * vy; }
                    else corr = hx ? vx : vy;
                    g.U[c] += T(1.0) * corr; } }
        };
        std::function<void(int)> cycle = [&](int d) {
            if (d == 0) { smooth(0, 0); return; }
            for (int s = 0; s < nu; ++s) { smooth(d, 0); smooth(d, 1); }
            restrict_(d);
            for (int k = 0; k < (d == 1 ? 1 : mu); ++k) cycle(d - 1);
            prolong(d);
            for (int s = 0; s < nu; ++s) { smooth(d, 0); smooth(d, 1); }
        };
        for (int call = 0; call < 2; ++call) cycle(dl);
        // ---- compare every node of every grid
        for (int g = 0; g < D.ngrid; ++g) {
            int w = D.grid[g], p = w & 15, q = (w >> 4) & 15, o = w >> 8;
            Grid& gr = G[p][q];
            for (int k = 0; k < (int)gr.U.size(); ++k) {
                ++checked;
                if (memcmp(&gr.U[k], &u[o + k], sizeof(T)) != 0) { if (bad < 10) printf("diff mu%d nu%d cls %d %d %d grid %d %d node %d: %g vs %g\n", mu, nu, pic, qic, dl, p, q, k, gr.U[k], u[o + k]); bad++; }
            }
        }
    }
    printf("program: %d node values compared, %d differ\n", checked, bad);
    return bad;
}

int main() { return (check_bounds() + check_program()) != 0; }
