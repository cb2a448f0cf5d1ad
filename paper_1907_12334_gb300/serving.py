"""Continuous-batching request loop fed by the adaptive MSG-MIMC driver.

``MimcDriver`` is Algorithm 3 of arXiv:1907.12334 (Sec. 3): it draws the
multi-index L^(n) of each sample from pi_L (initially the product of
geometric laws with r_j = log(2)(beta_j + gamma_j)/2, beta = 4, gamma = 1),
turns the FMSG solution of a sample into Y^(n) = sum_{0 <= tau <= L} dQ_tau /
p_tau (Eq. (3.6)), keeps E and V (Eqs. (3.7)-(3.8)) and re-estimates pi_L from
the running sqrt(V_l / C_l) of the differences (Eq. (3.10)), until sqrt(V) <= eps.

``Server`` takes sample requests as they arrive, admits them while their
device memory (field + solver workspace, from ``msg_workspace_bytes``) fits an
HBM budget, and runs admitted requests in batches on several CUDA streams at
once: a request that arrives while other batches are on the GPU is started in
the next free slot instead of waiting for the whole job.  KL bases are
prepared once per grid shape and stay on the device; xi, Z, the hierarchy and
the results of a batch live on the device until the batch finishes.  Each
request's latency is measured from its arrival to the moment its result is on
the host.  All arithmetic runs in the CUDA library; this module schedules.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------------ driver --

def geometric_tail(r, n):
    """P(L_j >= k) = exp(-r k), k = 0..n-1 (Algorithm 3's initial law, one axis)."""
    return np.exp(-r * np.arange(n))


@dataclass
class MimcDriver:
    """Algorithm 3 (MSG-MIMC) bookkeeping on the host.

    Indices are l = (p - p0, q - q0) with 0 <= l_j <= lmax_j (a memory cap in
    the spirit of the Sec. 4 remark on the index (0, 19))."""
    eps: float
    p0: int = 2
    q0: int = 2
    lmax: tuple = (6, 6)
    seed: int = 0
    beta: float = 4.0
    gamma: float = 1.0
    learn_every: int = 64
    n: int = 0
    Ysum: float = 0.0
    Y2sum: float = 0.0
    rng: np.random.Generator = field(init=False)

    def __post_init__(self):
        self.rng = np.random.default_rng(self.seed)
        r = 0.5 * math.log(2.0) * (self.beta + self.gamma)
        n1, n2 = self.lmax[0] + 1, self.lmax[1] + 1
        self.tail = np.outer(geometric_tail(r, n1), geometric_tail(r, n2))  # p_tau = P(L >= tau)
        self.sdq = np.zeros((n1, n2))
        self.sdq2 = np.zeros((n1, n2))
        self.cnt = np.zeros((n1, n2))
        self.skipped: dict[str, np.ndarray] = {}  # reason -> per-index count of samples without a Y
        self.cost = np.array([[2.0 ** ((self.p0 + a) + (self.q0 + b)) for b in range(n2)] for a in range(n1)])
        self.csum = np.zeros((n1, n2))  # measured work of the solves drawn at each index
        self.ccnt = np.zeros((n1, n2))

    def pmf(self):
        """pi_L from the tail probabilities: P(L = l) by inclusion-exclusion."""
        t = np.pad(self.tail, ((0, 1), (0, 1)))
        return t[:-1, :-1] - t[1:, :-1] - t[:-1, 1:] + t[1:, 1:]

    def draw(self, k):
        p = self.pmf().ravel()
        p = np.clip(p, 0, None)
        p /= p.sum()
        idx = self.rng.choice(p.size, size=k, p=p)
        n2 = self.lmax[1] + 1
        return [(int(i // n2), int(i % n2)) for i in idx]

    def shape(self, L):
        return (self.p0 + L[0], self.q0 + L[1])

    def record(self, L, dQ, ptau_used, cost=None):
        """dQ: [(L1+1), (L2+1)] differences of one sample; ptau_used: the p_tau at draw time;
        cost: the measured work of the sample's solve (replaces the prior C_l of its index)."""
        Y = float((dQ / ptau_used[: L[0] + 1, : L[1] + 1]).sum())
        if cost is not None and cost > 0:
            self.csum[L[0], L[1]] += cost
            self.ccnt[L[0], L[1]] += 1
        self.n += 1
        self.Ysum += Y
        self.Y2sum += Y * Y
        a, b = L[0] + 1, L[1] + 1
        self.sdq[:a, :b] += dQ
        self.sdq2[:a, :b] += dQ * dQ
        self.cnt[:a, :b] += 1
        if self.n % self.learn_every == 0:
            self.learn()
        return Y

    def take(self, req):
        """Fold one finished request into the estimator (record) or the skip counts."""
        if req.status == 0 and req.dQ is not None:
            return self.record(req.L, req.dQ, req.ptau, req.cost or None)
        self.skip(req.L, req.status)
        return None

    def skip(self, L, status):
        """Count a sample that gives no Y: its solve did not converge or became
        non-finite, its batch failed, or it was refused.  Leaving such samples out
        reweights Eq. (3.6) towards the indices that converge, so the counts are
        reported beside E and V (``skipped_report``)."""
        if status < 0:
            key = "refused" if status == -1 else "batch_failed"
        elif status & 2:
            key = "nonfinite"
        else:
            key = "not_converged"
        self.skipped.setdefault(key, np.zeros_like(self.cnt))[L[0], L[1]] += 1

    def skipped_report(self):
        """{reason: {(l1, l2): count}} of the samples left out of E and V."""
        return {k: {(int(a), int(b)): int(v[a, b]) for a, b in zip(*np.nonzero(v))} for k, v in self.skipped.items()}

    def learn(self):
        """Tail probabilities proportional to sqrt(V_l / C_l), normalised to p_0 = 1 and made
        monotone (READING of 'update the probability mass function' in Algorithm 3)."""
        with np.errstate(invalid="ignore", divide="ignore"):
            m = self.sdq / np.maximum(self.cnt, 1)
            v = self.sdq2 / np.maximum(self.cnt, 1) - m * m
        ok = self.cnt >= 8
        if not ok[0, 0]:
            return
        # C_l: measured mean work where solves at that index have been timed, else the prior
        # 2^(p+q) rescaled to the measured ones (Algorithm 3 updates pi_L from estimates)
        cost = self.cost.copy()
        seen = self.ccnt > 0
        if seen.any():
            mc = self.csum[seen] / self.ccnt[seen]
            scale = float(np.exp(np.mean(np.log(mc / self.cost[seen]))))
            cost = np.where(seen, self.csum / np.maximum(self.ccnt, 1), self.cost * scale)
        w = np.where(ok, np.sqrt(np.maximum(v, 0) / cost), 0.0)
        if w[0, 0] <= 0:
            return
        t = w / w[0, 0]
        t = np.where(ok, t, self.tail)  # keep the prior where there is no estimate
        # monotone non-increasing in both directions (a tail probability)
        t = np.minimum.accumulate(np.minimum.accumulate(t, axis=0), axis=1)
        self.tail = np.clip(t, 1e-12, 1.0)
        self.tail[0, 0] = 1.0

    @property
    def E(self):
        return self.Ysum / max(self.n, 1)

    @property
    def V(self):
        if self.n < 2:
            return float("inf")
        m = self.E
        return max(self.Y2sum / self.n - m * m, 0.0) * self.n / (self.n - 1) / self.n

    def done(self):
        return self.n >= 2 and math.sqrt(self.V) <= self.eps


def measured_cost(cycles):
    """Work of one FMSG solve from the cycles each grid used: a mu-cycle of Algorithm 1
    with grid (p,q) as its top visits every grid of its hierarchy about once per
    finest-grid unknown (Sec. 2), so a cycle costs ~ p q 2^(p+q) unknown updates."""
    P, Q = cycles.shape
    p = np.arange(1, P + 1)[:, None]
    q = np.arange(1, Q + 1)[None, :]
    return float((cycles * p * q * np.exp2(p + q)).sum())


# ------------------------------------------------------------------ server --

STATUS_REFUSED = -1       # request larger than the whole HBM budget
STATUS_BATCH_FAILED = -2  # the batch's library call raised; Q and dQ are None

@dataclass
class Request:
    rid: int
    sample: int      # global sample number (the xi counter)
    L: tuple
    shape: tuple
    ptau: np.ndarray
    t_arrive: float = 0.0
    t_done: float = 0.0
    Q: np.ndarray | None = None
    dQ: np.ndarray | None = None
    status: int = 0  # MSG_SAMPLE_* bits of the solve, or STATUS_REFUSED / STATUS_BATCH_FAILED
    error: str = ""
    cost: float = 0.0  # measured work of the solve (see measured_cost)


class Server:
    """Continuous batching of FMSG sample requests on one GPU."""

    def __init__(self, hbm_budget_bytes: int, max_batch: int = 1024, slots: int = 3, M: int = 64, seed: int = 0,
                 prm=None, p0: int = 2, q0: int = 2, device="cuda:0"):
        import torch

        from . import build, inputs, msg

        build.build()
        msg.load()
        self.torch, self.msg, self.inputs = torch, msg, inputs
        self.dev = torch.device(device)
        self.budget = int(hbm_budget_bytes)
        self.max_batch = max_batch
        self.M, self.seed, self.p0, self.q0 = M, seed, p0, q0
        self.prm = prm or msg.SolverParams()
        self.law = inputs.FieldLaw(M=M)
        self.bases = {}  # (P, Q) -> (prepared, npts): device-resident KL bases
        self.lock = threading.Lock()
        self.inbox: "queue.Queue[Request]" = queue.Queue()
        self.in_use = 0
        self.done: list[Request] = []
        self.rejected = 0
        self.failures: list[str] = []
        self.slots = slots
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.busy = [False] * slots
        self.cv = threading.Condition()
        self.batches = 0

    # -------------------------------------------------------------- basis --
    def basis(self, P, Q):
        with self.lock:
            if (P, Q) not in self.bases:
                Phi, sl = self.inputs.kl_basis(P, Q, self.law)
                npts = Phi.shape[0]
                m = self.msg.MSG_GEMM_FP64
                prep = self.torch.empty(self.msg.kl_prepared_bytes(npts, self.M, m), dtype=self.torch.uint8,
                                        device=self.dev)
                self.msg.kl_prepare(self.torch.from_numpy(np.ascontiguousarray(Phi)).to(self.dev),
                                    self.torch.from_numpy(np.array(sl)).to(self.dev), m, prep)
                self.torch.cuda.synchronize(self.dev)
                self.bases[(P, Q)] = (prep, npts)
            return self.bases[(P, Q)]

    def request_bytes(self, shapes):
        pq = np.array(shapes, dtype=np.int32).reshape(-1, 2)
        nf = sum(self.msg.field_points(int(a), int(b)) for a, b in pq)
        return self.msg.msg_workspace_bytes(pq, self.prm) + 8 * nf + 8 * len(shapes) * self.M

    # ------------------------------------------------------------ running --
    def submit(self, req: Request):
        req.t_arrive = time.perf_counter()
        self.inbox.put(req)

    def _run_batch(self, slot, reqs):
        torch, msg = self.torch, self.msg
        st = self.streams[slot]
        try:
            with torch.cuda.stream(st):
                S = len(reqs)
                shapes = np.array([r.shape for r in reqs], dtype=np.int32)
                nq, nf = msg.packed_sizes(shapes)
                Z = torch.empty(nf, dtype=torch.float64, device=self.dev)
                foff = np.concatenate([[0], np.cumsum([msg.field_points(*r.shape) for r in reqs])])
                # fields: one KL contraction per shape group of the batch (each group's basis
                # stays on the device), then placed at the requests' offsets
                groups = {}
                for k, r in enumerate(reqs):
                    groups.setdefault(tuple(r.shape), []).append(k)
                for shape, ks in groups.items():
                    prep, npts = self.basis(*shape)
                    xi = torch.empty((len(ks), self.M), dtype=torch.float64, device=self.dev)
                    for j, k in enumerate(ks):
                        msg.msg_normals(self.seed, reqs[k].sample, 1, self.M, xi[j:j + 1], stream=st)
                    Zs = torch.empty((len(ks), npts), dtype=torch.float64, device=self.dev)
                    msg.sample_field(prep, npts, self.M, msg.MSG_GEMM_FP64, xi, Zs, stream=st)
                    for j, k in enumerate(ks):
                        Z[int(foff[k]):int(foff[k + 1])].copy_(Zs[j])
                Q = torch.empty(nq, dtype=torch.float64, device=self.dev)
                status = torch.empty(S, dtype=torch.int32, device=self.dev)
                cyc = torch.empty(nq, dtype=torch.int32, device=self.dev)
                ws = torch.empty(msg.msg_workspace_bytes(shapes, self.prm), dtype=torch.uint8, device=self.dev)
                msg.msg_solve_batch(shapes, self.prm, Z, Q, status, cycles=cyc, workspace=ws, stream=st)
                Ls = np.array([r.L for r in reqs], dtype=np.int32)
                nd = int(sum((a + 1) * (b + 1) for a, b in Ls))
                dQ = torch.empty(nd, dtype=torch.float64, device=self.dev)
                msg.mimc_differences(Ls, self.p0, self.q0, Q, dQ, stream=st)
                st.synchronize()
                Qh, dQh, sth, cych = Q.cpu().numpy(), dQ.cpu().numpy(), status.cpu().numpy(), cyc.cpu().numpy()
            t = time.perf_counter()
            oq = od = 0
            for k, r in enumerate(reqs):
                P, Qn = r.shape
                r.Q = Qh[oq:oq + P * Qn].reshape(P, Qn)
                r.cost = measured_cost(cych[oq:oq + P * Qn].reshape(P, Qn))
                oq += P * Qn
                a, b = r.L[0] + 1, r.L[1] + 1
                r.dQ = dQh[od:od + a * b].reshape(a, b)
                od += a * b
                r.status = int(sth[k])
                r.t_done = t
        except Exception as exc:  # a library or allocation failure fails the whole batch, visibly
            t = time.perf_counter()
            for r in reqs:
                r.status = STATUS_BATCH_FAILED
                r.Q = r.dQ = None
                r.error = repr(exc)
                r.t_done = t
            self.failures.append(repr(exc))
        finally:
            with self.cv:
                self.in_use -= self.request_bytes([r.shape for r in reqs])
                self.busy[slot] = False
                self.done.extend(reqs)
                self.batches += 1
                self.cv.notify_all()

    def start(self):
        """Run the admission loop on a background thread until stop()."""
        self._stop = threading.Event()
        self._threads = []
        self._loop_thread = threading.Thread(target=self._loop, daemon=True)
        self._loop_thread.start()
        return self

    def stop(self):
        self._stop.set()
        self._loop_thread.join()
        for th in self._threads:
            th.join()

    def _loop(self):
        pending: list[Request] = []
        while not self._stop.is_set():
            try:
                while True:
                    pending.append(self.inbox.get_nowait())
            except queue.Empty:
                pass
            with self.cv:
                free = [i for i in range(self.slots) if not self.busy[i]]
                if not free or not pending:
                    self.cv.wait(timeout=0.002)
                    continue
                # admission by HBM budget, first come first served
                batch, need = [], 0
                for r in list(pending):
                    cand = batch + [r]
                    nb = self.request_bytes([x.shape for x in cand])
                    if self.in_use + nb > self.budget or len(cand) > self.max_batch:
                        if not batch and self.in_use == 0:
                            self.rejected += 1  # a single request above the budget: refused
                            pending.remove(r)
                            r.status = STATUS_REFUSED
                            r.t_done = time.perf_counter()
                            self.done.append(r)
                        break
                    batch, need = cand, nb
                if not batch:
                    self.cv.wait(timeout=0.002)
                    continue
                for r in batch:
                    pending.remove(r)
                slot = free[0]
                self.busy[slot] = True
                self.in_use += need
            th = threading.Thread(target=self._run_batch, args=(slot, batch), daemon=True)
            th.start()
            self._threads.append(th)

    def serve(self, requests, timeout: float = 3600.0):
        """Submit `requests` at once and return them when all are done."""
        self.start()
        for r in requests:
            self.submit(r)
        t_end = time.perf_counter() + timeout
        with self.cv:
            while len(self.done) < len(requests):
                if time.perf_counter() > t_end:
                    break
                self.cv.wait(timeout=0.01)
        self.stop()
        return list(self.done)

    @staticmethod
    def latency_stats(done):
        lat = np.array([r.t_done - r.t_arrive for r in done]) * 1000.0
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "n": int(lat.size)}


def run_driver(server: Server, driver: MimcDriver, rate_hz: float, max_samples: int, seed: int = 1):
    """Feed the server with Poisson arrivals of driver requests until sqrt(V) <= eps
    (or max_samples); returns (driver, results, wall seconds).  Samples without a
    usable result are counted per multi-index in ``driver.skipped_report()``."""
    rng = np.random.default_rng(seed)
    results = []
    sent = 0
    t0 = time.perf_counter()
    feeder_done = threading.Event()

    def feeder():
        nonlocal sent
        while sent < max_samples and not driver.done():
            L = driver.draw(1)[0]
            req = Request(rid=sent, sample=sent, L=L, shape=driver.shape(L), ptau=driver.tail.copy())
            server.submit(req)
            sent += 1
            time.sleep(rng.exponential(1.0 / rate_hz))
        feeder_done.set()

    server.start()
    th = threading.Thread(target=feeder, daemon=True)
    th.start()
    seen = 0
    while True:
        with server.cv:
            fresh = server.done[seen:]
            seen = len(server.done)
        for r in fresh:
            driver.take(r)
            results.append(r)
        if feeder_done.is_set() and seen >= sent:
            break
        time.sleep(0.002)
    server.stop()
    return driver, results, time.perf_counter() - t0
