"""Differentiable chunked diffusion: forward and adjoint annotated launches
behind a torch.autograd.Function (an extension beyond the paper).

    u_{t+1} = u_t + kappa * (L u_t),   (L u)_ij = u_{i-1,j} + u_{i+1,j} + u_{i,j-1} + u_{i,j+1} - 4 u_ij

The forward pass keeps a checkpoint of u every ``ckpt`` steps.  The backward
pass walks the segments backwards: it recomputes the states of a segment
from its checkpoint, then runs one adjoint launch per step, whose
annotation is the forward one transposed (the halo read of u becomes a
halo reduce(+) of lambda):

    lambda_t = lambda_{t+1} + L(kappa * lambda_{t+1})
    dkappa  += lambda_{t+1} * (L u_t)

and returns dJ/du0 = lambda_0 and dJ/dkappa.  The incoming gradient
grad_output is lambda_T (for J = sum u_T^2 it is 2 u_T).  With
ckpt_every = 1 every state is kept and nothing is recomputed (one forward
and one adjoint launch per step).

PyTorch only moves the fields between tensors and the engine's arrays
(device-to-device copies); every step runs in the engine's kernels.
"""
from __future__ import annotations

import torch

from . import _lib as L
from . import lightning as lt

FWD_ANN = "global [i, j] => read U[i-1:i+1, j-1:j+1], read K[i, j], write V[i, j]"
ADJ_ANN = ("global [i, j] => read L1[i, j], read K[i, j], read U[i-1:i+1, j-1:j+1], readwrite G[i, j], "
           "reduce(+) L0[i-1:i+1, j-1:j+1]")


class DiffusionPlan:
    """Arrays and kernels for `steps` diffusion steps on an ny x nx grid,
    chunked by `dist`, launched in superblocks of `superblock` threads."""

    def __init__(self, ctx: lt.Context, ny: int, nx: int, steps: int, ckpt: int, dist: lt.Dist, superblock):
        assert steps >= 1 and ckpt >= 1
        self.ctx, self.ny, self.nx, self.steps, self.ckpt = ctx, ny, nx, steps, ckpt
        self.sb = tuple(superblock)
        self.segs = [(s, min(ckpt, steps - s)) for s in range(0, steps, ckpt)]
        mk = lambda: ctx.array(lt.F32, (ny, nx), dist)  # noqa: E731
        self.K = mk()
        self.ck = [mk() for _ in range(len(self.segs) + 1)]
        self.work = [mk() for _ in range(max(1, ckpt - 1))]
        self.lam = [mk(), mk()]
        self.G = mk()
        self.kf = ctx.kernel(lt.DIFFUSION2D, FWD_ANN, [("U", lt.F32), ("K", lt.F32), ("V", lt.F32)])
        self.ka = ctx.kernel(lt.DIFFUSION2D_ADJ, ADJ_ANN, [("L1", lt.F32), ("K", lt.F32), ("U", lt.F32),
                                                           ("G", lt.F32), ("L0", lt.F32)])

    def arrays(self):
        return [self.K, self.G] + self.ck + self.work + self.lam

    def release(self):
        """Give the arrays and kernels back to the context."""
        if self.K is None:
            return
        for a in self.arrays():
            a.destroy()
        self.kf.destroy()
        self.ka.destroy()
        self.K = None

    def __del__(self):
        try:
            if self.K is not None and self.ctx.h:
                self.release()
        except Exception:
            pass

    def _fwd(self, src, dst):
        self.kf.launch(grid=(self.nx, self.ny), block=(128, 2), superblock=self.sb, args=[src, self.K, dst])

    def _adj(self, l1, u, l0):
        self.ka.launch(grid=(self.nx, self.ny), block=(128, 2), superblock=self.sb, args=[l1, self.K, u, self.G, l0])

    def forward(self):
        """u_T into ck[-1]; checkpoints at the start of every segment."""
        for k, (s, n) in enumerate(self.segs):
            cur = self.ck[k]
            for j in range(n):
                dst = self.ck[k + 1] if j == n - 1 else self.work[j]
                self._fwd(cur, dst)
                cur = dst

    def backward(self):
        """lambda_T must be in lam[0]; leaves dJ/du0 in the returned array and dJ/dkappa in G."""
        self.G.fill(L.LT_INIT_ZERO)
        cur, nxt = self.lam
        for k in reversed(range(len(self.segs))):
            s, n = self.segs[k]
            states = [self.ck[k]]
            for j in range(1, n):  # recompute u_{s+1} .. u_{s+n-1} from the checkpoint
                self._fwd(states[-1], self.work[j - 1])
                states.append(self.work[j - 1])
            for j in reversed(range(n)):
                self._adj(cur, states[j], nxt)
                cur, nxt = nxt, cur
        return cur


_ctx_cache: dict = {}
_plan_cache: dict = {}  # (context, shape, steps, ckpt, chunk, superblock) -> idle DiffusionPlans


def _context(device: int, budget: int) -> lt.Context:
    key = (device, budget)
    if key not in _ctx_cache:
        _ctx_cache[key] = lt.Context(device=device, hbm_budget=budget)
    return _ctx_cache[key]


def _plan(ectx, ny, nx, steps, ckpt, chunk, superblock, dist):
    """An idle plan of this shape (its arrays and kernels are kept between
    calls: creating 19 arrays and registering two kernels per call cost
    host time the GPU waited for), or a new one."""
    key = (id(ectx), ny, nx, steps, ckpt, chunk, tuple(superblock))
    idle = _plan_cache.setdefault(key, [])
    return idle.pop() if idle else DiffusionPlan(ectx, ny, nx, steps, ckpt, dist, superblock), key


def clear_caches():
    """Release the cached plans and contexts (their HBM pools)."""
    for plans in _plan_cache.values():
        for p in plans:
            p.release()
    _plan_cache.clear()
    for c in _ctx_cache.values():
        c.close()
    _ctx_cache.clear()


class DiffusionChunked(torch.autograd.Function):
    """u_T = DiffusionChunked.apply(u0, kappa, steps, ckpt_every, chunk, superblock).

    u0 and kappa: contiguous f32 CUDA tensors of shape (ny, nx).  chunk: tile
    extent of the distribution (0 = one chunk), halo 1; superblock: threads
    per superblock (x, y), 0 = whole grid."""

    @staticmethod
    def forward(ctx, u0, kappa, steps: int, ckpt_every: int = 10, chunk: int = 0, superblock=(0, 0)):
        assert u0.is_cuda and u0.dtype == torch.float32 and kappa.shape == u0.shape
        ny, nx = u0.shape
        field = ny * nx * 4
        nfields = (steps + ckpt_every - 1) // ckpt_every + 1 + max(1, ckpt_every - 1) + 4
        budget = int(nfields * field * 1.15 + field * 2.5) + (256 << 20)
        ectx = _context(u0.device.index or 0, budget)
        dist = lt.Dist.tiles((chunk, chunk), halo=(1, 1)) if chunk else lt.Dist.block()
        plan, key = _plan(ectx, ny, nx, steps, ckpt_every, chunk, superblock, dist)
        u0c, kc = u0.detach().contiguous(), kappa.detach().contiguous()
        torch.cuda.synchronize(u0.device)
        plan.K.write_device(kc.data_ptr(), field)
        plan.ck[0].write_device(u0c.data_ptr(), field)
        plan.forward()
        out = torch.empty_like(u0c)
        plan.ck[-1].read_device(out.data_ptr(), field)
        ctx.plan = plan
        ctx.plan_key = key
        return out

    @staticmethod
    def backward(ctx, grad_out):
        plan: DiffusionPlan = ctx.plan
        field = plan.ny * plan.nx * 4
        g = grad_out.detach().to(torch.float32).contiguous()
        torch.cuda.synchronize(g.device)
        plan.lam[0].write_device(g.data_ptr(), field)
        lam0 = plan.backward()
        du0 = torch.empty_like(g)
        dk = torch.empty_like(g)
        lam0.read_device(du0.data_ptr(), field)
        plan.G.read_device(dk.data_ptr(), field)
        _plan_cache.setdefault(ctx.plan_key, []).append(plan)  # idle again: the next call of this shape reuses it
        ctx.plan = None
        return du0, dk, None, None, None, None
