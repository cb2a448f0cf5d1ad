// Host check of the low-diagonal tables built by solver.cu (no GPU needed):
//  1. every shared-memory index that any table entry of any class can produce
//     lies inside that plane of the class's layout, and the zero slot is never
//     written;
//  2. each class's resolved program, run on the planes through the kernel's own
//     per-node functions (their host builds) for several items side by side in
//     one strided buffer, with table phases throughout and with the register path
//     below diagonal 3, gives bit for bit the values of a plain recursive
//     W-cycle of Algorithm 1 (with the same two program simplifications: the
//     restriction clears the child's correction, and diagonal 0 is solved once
//     per diagonal-1 visit) run on full node arrays of every grid.
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
    auto in = [&](long v, long n, const char* w, int pic, int qic, int dl) {
        if (v < 0 || v >= n) { if (bad < 20) printf("OOB %s %ld/%ld cls %d %d %d\n", w, v, n, pic, qic, dl); bad++; }
    };
    for (int dl = 0; dl <= kLowMax; ++dl) {
        const LowPlanes& L = lt.planes[dl];
        for (int pic = 1; pic <= dl + 1; ++pic)
            for (int qic = 1; qic <= dl + 1; ++qic) {
                const LowDesc& D = lt.desc[low_class(pic, qic, dl)];
                if (D.dl != dl || D.pic != pic || D.qic != qic) { printf("class index\n"); bad++; }
                for (int d = 0; d <= dl; ++d)
                    for (int kd = 0; kd < LK_NKIND; ++kd)
                        if (D.cnt[d][kd] && (D.off[d][kd] < D.e0 || D.off[d][kd] + D.cnt[d][kd] > D.e1)) {
                            printf("entries outside the class range\n"); bad++; }
                auto node = [&](uint4 e, bool resid) {
                    int c = e.x & 0xFFFF, uw = e.x >> 16, ue = e.y & 0xFFFF, us = e.y >> 16, un = e.z & 0xFFFF;
                    int xw = e.z >> 16, ys = e.w & 0xFFFF, r = e.w >> 16;
                    if (c == 0) { printf("writes the zero slot\n"); bad++; }
                    for (int v : {c, uw, ue, us, un}) in(v, L.nu, "u", pic, qic, dl);
                    in(xw, L.nfx, "fx", pic, qic, dl); in(xw + 1, L.nfx, "fx", pic, qic, dl);
                    in(ys, L.nfy, "fy", pic, qic, dl); in(ys + 1, L.nfy, "fy", pic, qic, dl);
                    if (resid) in(r, L.nr, "r", pic, qic, dl);
                };
                for (int d = 0; d <= dl; ++d) {
                    for (int k = 0; k < 2; ++k)
                        for (int e = 0; e < D.cnt[d][k]; ++e) node(lt.ent[D.off[d][k] + e], d > 0);
                    if (D.off[d][LK_RESID] != D.off[d][LK_RED] ||
                        D.cnt[d][LK_RESID] != D.cnt[d][LK_RED] + D.cnt[d][LK_BLACK] ||
                        D.off[d][LK_BLACK] != D.off[d][LK_RED] + D.cnt[d][LK_RED]) { printf("resid list\n"); bad++; }
                    for (int e = 0; e < D.cnt[d][LK_RESTRICT]; ++e) {
                        uint4 a = lt.ent[D.off[d][LK_RESTRICT] + e];
                        int c = a.x & 0xFFFF, rx = a.x >> 16, ry = a.y & 0xFFFF, wy = a.y >> 16;
                        bool hx = a.z & 1, hy = a.z & 2;
                        in(c, L.nu, "cu", pic, qic, dl);
                        if (c == 0) { printf("restrict writes the zero slot\n"); bad++; }
                        if (!hx && !hy) { printf("no parent\n"); bad++; }
                        if (hx) for (int s = -1; s <= 1; ++s) in(rx + s, L.nr, "rx", pic, qic, dl);
                        if (hy) for (int s = -1; s <= 1; ++s) in(ry + s * wy, L.nr, "ry", pic, qic, dl);
                    }
                    for (int e = 0; e < D.cnt[d][LK_PROL]; ++e) {
                        uint4 v = lt.ent[D.off[d][LK_PROL] + e];
                        int c = v.x & 0xFFFF, xw = v.x >> 16, ys = v.y & 0xFFFF;
                        in(c, L.nu, "pc", pic, qic, dl);
                        if (c == 0) { printf("prolong writes the zero slot\n"); bad++; }
                        in(xw, L.nfx, "pfx", pic, qic, dl); in(xw + 1, L.nfx, "pfx", pic, qic, dl);
                        in(ys, L.nfy, "pfy", pic, qic, dl); in(ys + 1, L.nfy, "pfy", pic, qic, dl);
                        for (int ch : {(int)(v.y >> 16), (int)(v.z & 0xFFFF), (int)(v.z >> 16), (int)(v.w & 0xFFFF)})
                            in(ch, L.nu, "child", pic, qic, dl);
                    }
                }
            }
        // grid slots of the fixed layout tile the planes
        int nu = 1, nfx = 0, nfy = 0;
        for (int g = 0; g < L.ngrid; ++g) {
            const LowGrid& G = L.g[g];
            int nx = 1 << G.p, ny = 1 << G.q;
            if (G.gu != nu || G.gx != nfx || G.gy != nfy) { printf("layout\n"); bad++; }
            nu += (nx - 1) * (ny - 1); nfx += low_pad4(nx * (ny - 1)); nfy += low_pad4((nx - 1) * ny);
            if (g < 6 && (r2::gp(g) != G.p || r2::gq(g) != G.q || r2::gu(g) + 1 != G.gu || r2::gx(g) != G.gx ||
                          r2::gy(g) != G.gy)) { printf("register-path offsets\n"); bad++; }
            if (G.gx % 4 || G.gy % 4) { printf("face alignment\n"); bad++; }
            std::vector<int> seen((nx - 1) * (ny - 1), 0);
            for (int j = 1; j < ny; ++j)
                for (int i = 1; i < nx; ++i) seen[low_rb(nx - 1, ny - 1, i, j)]++;
            for (int v : seen) if (v != 1) { printf("rb order\n"); bad++; break; }
        }
        if (low_pad4(nu) != L.nu || nfx != L.nfx || nfy != L.nfy) { printf("plane sizes\n"); bad++; }
        if (dl > 0) {  // prefix property: the lower layout's grids keep their offsets
            const LowPlanes& Lm = lt.planes[dl - 1];
            for (int g = 0; g < Lm.ngrid; ++g)
                if (Lm.g[g].gu != L.g[g].gu || Lm.g[g].gx != L.g[g].gx || Lm.g[g].gy != L.g[g].gy) { printf("prefix\n"); bad++; }
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
                    if (kind == LK_CALL2) { if (D.dl < 3) bad++; continue; }
                    if (kind >= LK_NKIND || cnt <= 0 || off < 0 || D.e0 + off + cnt > D.e1) bad++;
                }
        }
    // shared-memory layout of a launch: entries, program, then the items' planes; the
    // face planes of every item must start 16-byte aligned (they are filled by 16-byte copies)
    for (int prec = 0; prec <= 1; ++prec)
        for (int mu = 1; mu <= 3; ++mu)
            for (int nu = 1; nu <= 3; ++nu) {
                msg_params prm{}; prm.mu = mu; prm.nu1 = nu; prm.nu2 = nu; prm.precision = prec;
                const size_t es = prec == MSG_PREC_MIXED ? 4 : 8;
                for (int kw : {1, 2, 4, 8})
                    for (int wpb : {1, 3, 8, 16}) {
                        const LowShape sh = low_shape_at(prm, kLowMax, kw, wpb);
                        for (int dl = 0; dl <= kLowMax; ++dl) {
                            const LowPlanes& L = lt.planes[dl];
                            const int stride = low_stride(L, kw, es);
                            const size_t base = 16 * (size_t)sh.ecap[dl] + 8 * (size_t)sh.pcap[dl];
                            for (int w = 0; w < wpb; ++w)
                                for (int k = 0; k < kw; ++k) {
                                    const size_t u0 = base + es * (size_t)(w * kw + k) * stride;
                                    const size_t fx0 = u0 + es * 2 * L.nu, fy0 = fx0 + es * L.nfx;
                                    if (fx0 % 16 || fy0 % 16 || base % 16) { if (bad < 20) printf("smem alignment\n"); bad++; }
                                }
                            if (sh.smem[dl] != base + es * (size_t)stride * kw * wpb) { printf("smem size\n"); bad++; }
                            if ((L.nfx * es) % 16 || (L.nfy * es) % 16) { printf("plane size\n"); bad++; }
                        }
                        const LowPlanes& L5 = lt.planes[kLowMax];
                        if (((L5.nfx + L5.nfy) * es) % 16 || (L5.nfx * es) % 16) { printf("image stride\n"); bad++; }
                    }
            }
    printf("bounds: %zu table entries, %d out of range\n", lt.ent.size(), bad);
    return bad;
}

static int check_program()
{
    const LowTables& lt = low_tables();
    std::mt19937 rng(1);
    std::uniform_real_distribution<float> ud(0.05f, 3.0f), ub(-1.f, 1.f);
    int bad = 0, checked = 0;
    const int KW = 3;  // items side by side in one strided buffer, as a warp holds them
    for (int reg2 = 0; reg2 <= 1; ++reg2)  // table phases throughout, and the register path below diagonal 3
    for (int mu = 1; mu <= 3; ++mu)
    for (int nu = 1; nu <= 2; ++nu)
    for (int dl = 0; dl <= kLowMax; ++dl)
    for (int pic = 1; pic <= dl + 1; ++pic)
    for (int qic = 1; qic <= dl + 1; ++qic) {
        if (pic + qic < dl + 2) continue;  // no item has such a class
        if (dl == kLowMax && mu == 3) continue;  // keeps the host run short; mu = 3 is covered below kLowMax
        msg_params prm{}; prm.mu = mu; prm.nu1 = nu; prm.nu2 = nu; prm.omega = 1.0; prm.precision = MSG_PREC_MIXED;
        std::vector<LowDesc> desc;
        std::vector<uint2> rp = low_resolve(prm, desc, reg2 != 0);
        const LowDesc& D = desc[low_class(pic, qic, dl)];
        const LowPlanes& L = lt.planes[dl];
        const int stride = low_stride(L, 4, sizeof(T));
        auto exists = [&](int p, int q) { return p >= 1 && q >= 1 && p <= pic && q <= qic && p + q - 2 <= dl; };
        std::vector<T> buf((size_t)stride * KW, -777.f);
        std::vector<std::vector<std::vector<Grid>>> GI(KW, std::vector<std::vector<Grid>>(8, std::vector<Grid>(8)));
        for (int it = 0; it < KW; ++it) {
            auto& G = GI[it];
            for (int p = 1; p <= 7; ++p) for (int q = 1; q <= 7; ++q) if (exists(p, q)) {
                Grid& g = G[p][q]; g.p = p; g.q = q; g.nx = 1 << p; g.ny = 1 << q; g.W = g.nx + 1;
                int n = (g.nx + 1) * (g.ny + 1);
                g.U.assign(n, 0.f); g.B.assign(n, 0.f); g.AX.resize(n); g.AY.resize(n);
                for (auto& v : g.AX) v = ud(rng);
                for (auto& v : g.AY) v = ud(rng);
                if (p + q - 2 == dl) for (int j = 1; j < g.ny; ++j) for (int i = 1; i < g.nx; ++i) g.B[j * g.W + i] = ub(rng);
            }
            // ---- planes filled like the kernel's prologue
            T* u = buf.data() + (size_t)it * stride; T* b = u + L.nu; T* fx = b + L.nu; T* fy = fx + L.nfx;
            if (2 * L.nu + L.nfx + L.nfy + L.nr > stride) { printf("stride too small\n"); bad++; }
            for (int k = 0; k < L.nu; ++k) u[k] = 0;
            for (int gi = 0; gi < L.ngrid; ++gi) {
                const LowGrid& LG = L.g[gi];
                int p = LG.p, q = LG.q;
                if (p > pic || q > qic) continue;
                int nx = 1 << p, ny = 1 << q, W = nx + 1;
                Grid& gr = G[p][q];
                for (int v = 0; v < ((ny - 1) << p); ++v) { int i = v & (nx - 1), j = 1 + (v >> p); fx[LG.gx + v] = gr.AX[j * W + i]; }
                for (int v = 0; v < (ny << p); ++v) { int i = v & (nx - 1), j = v >> p; if (!i) continue; fy[LG.gy + (i - 1) * ny + j] = gr.AY[j * W + i]; }
                if (p + q - 2 == dl)
                    for (int v = 0; v < ((ny - 1) << p); ++v) { int i = v & (nx - 1), j = 1 + (v >> p); if (!i) continue; b[LG.gu + low_rb(nx - 1, ny - 1, i, j)] = gr.B[j * W + i]; }
            }
        }
        // ---- the program, twice (two mu-cycles, as the kernel's calls = 2), each item in turn per phase
        for (int call = 0; call < 2; ++call)
            for (int o = 0; o < D.nops; ++o) {
                uint2 op = rp[D.prog + o]; int kind = op.x & 7, cnt = op.x >> 3, off = op.y;
                for (int it = 0; it < KW; ++it) {
                    T* u = buf.data() + (size_t)it * stride; T* b = u + L.nu; T* fx = b + L.nu; T* fy = fx + L.nfx;
                    T* r = fy + L.nfy;
                    if (kind == LK_CALL2) { low_call2(pic, qic, u, b, fx, fy, mu, nu, nu, (T)1.0); continue; }
                    for (int k = cnt - 1; k >= 0; --k)  // any order within a phase gives the same values
                        low_phase(kind, u, b, fx, fy, r, lt.ent[D.e0 + off + k], (T)1.0);
                }
            }
        for (int it = 0; it < KW; ++it) {
            auto& G = GI[it];
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
            // ---- compare every interior node of every grid, and the zero slot
            const T* u = buf.data() + (size_t)it * stride;
            if (u[0] != 0.f) { printf("zero slot written\n"); bad++; }
            for (int gi = 0; gi < L.ngrid; ++gi) {
                const LowGrid& LG = L.g[gi];
                int p = LG.p, q = LG.q;
                if (!exists(p, q)) continue;
                if (reg2 && dl >= 3 && p + q - 2 < 2) continue;  // those live in registers only
                Grid& gr = G[p][q];
                for (int j = 1; j < gr.ny; ++j)
                    for (int i = 1; i < gr.nx; ++i) {
                        ++checked;
                        T want = gr.U[j * gr.W + i], got = u[LG.gu + low_rb(gr.nx - 1, gr.ny - 1, i, j)];
                        if (memcmp(&want, &got, sizeof(T)) != 0) {
                            if (bad < 10) printf("diff mu%d nu%d cls %d %d %d grid %d %d node %d %d: %g vs %g\n", mu, nu, pic, qic, dl, p, q, i, j, want, got);
                            bad++;
                        }
                    }
            }
        }
    }
    printf("program: %d node values compared, %d differ\n", checked, bad);
    return bad;
}

int main() { return (check_bounds() + check_program()) != 0; }
