"""Torch-facing plan object and autograd functions over the C ABI.

PyTorch supplies device memory and streams only; every step of the transform
runs in libnfft_gb300.so.  Layout conventions are those of the C header:
f and y have shape N (row-major, index n_d + floor(N_d/2)), nodes k have
shape (M, D) in [-1/2, 1/2), fhat has shape (M,).

    plan = Plan((128, 128, 128), M, sigma=2.0, m=4, dtype=torch.complex64)
    plan.set_nodes(k)            # (M, 3) float64, device or host
    fhat = plan.forward(f)       # Algorithm 1
    y = plan.adjoint(fhat)       # Algorithm 2
    fhat = nfft(f, k, plan)      # differentiable in f and k
"""
import torch

from . import binding as B

_DTYPES = {torch.complex64: B.NFFT_C64, torch.complex128: B.NFFT_C128}
_REAL = {torch.complex64: torch.float32, torch.complex128: torch.float64}


def _ptr(t):
    return t.data_ptr() if t.numel() > 0 else 0


class Plan:
    """An NFFT plan (Sec. 3.1-3.2 of the paper): fixed N, M, sigma, m, dtype."""

    def __init__(self, N, M, sigma=2.0, m=4, dtype=torch.complex64, flags=0, stream=None,
                 device=None):
        if dtype not in _DTYPES:
            raise TypeError("dtype must be torch.complex64 or torch.complex128")
        self.N = tuple(int(v) for v in N)
        self.D = len(self.N)
        self.M = int(M)
        self.sigma = float(sigma)
        self.m = int(m)
        self.dtype = dtype
        self.real_dtype = _REAL[dtype]
        self.flags = int(flags)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            s, h = B.nfft_plan_create(self.D, self.N, self.M, self.sigma, self.m, _DTYPES[dtype],
                                      self.flags, self.stream.cuda_stream)
        B.check(s, "nfft_plan_create")
        self._h = h
        self._nodes_key = None

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            B.nfft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("plan is closed")
        return self._h

    # -- helpers ----------------------------------------------------------
    def _check_tensor(self, t, shape, dtype, name):
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch.Tensor" % name)
        if tuple(t.shape) != tuple(shape):
            raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
        if t.dtype != dtype:
            raise TypeError("%s has dtype %s, expected %s" % (name, t.dtype, dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.is_cuda and t.device != self.device:
            raise ValueError("%s is on %s, the plan on %s" % (name, t.device, self.device))

    def _out(self, out, shape, dtype, like):
        if out is None:
            dev = like.device if like is not None else self.device
            pin = not dev.type == "cuda"
            out = torch.empty(shape, dtype=dtype, device=dev, pin_memory=pin and torch.cuda.is_available())
        self._check_tensor(out, shape, dtype, "out")
        return out

    # -- API ---------------------------------------------------------------
    def set_nodes(self, k):
        """k: (M, D) float64 (preferred) or float32, device or host."""
        self._check_tensor(k, (self.M, self.D), k.dtype, "k")
        if k.dtype not in (torch.float64, torch.float32):
            raise TypeError("k must be float64 or float32")
        B.check(B.nfft_set_nodes(self.handle, _ptr(k), k.dtype == torch.float64), "nfft_set_nodes")
        self._nodes_key = (k.data_ptr(), k._version, k.device)

    def nodes_match(self, k):
        return self._nodes_key == (k.data_ptr(), k._version, k.device)

    def forward(self, f, out=None):
        """Direct NFFT (Algorithm 1): fhat = A f."""
        self._check_tensor(f, self.N, self.dtype, "f")
        out = self._out(out, (self.M,), self.dtype, f)
        B.check(B.nfft_forward(self.handle, _ptr(f), _ptr(out)), "nfft_forward")
        return out

    def adjoint(self, fhat, out=None):
        """Adjoint NFFT (Algorithm 2): y = A^H fhat."""
        self._check_tensor(fhat, (self.M,), self.dtype, "fhat")
        out = self._out(out, self.N, self.dtype, fhat)
        B.check(B.nfft_adjoint(self.handle, _ptr(fhat), _ptr(out)), "nfft_adjoint")
        return out

    def grad(self, f, cot, out=None):
        """gk[j, d] = Re(conj(cot_j) d(A f)_j / d k_{j,d})."""
        self._check_tensor(f, self.N, self.dtype, "f")
        self._check_tensor(cot, (self.M,), self.dtype, "cot")
        out = self._out(out, (self.M, self.D), self.real_dtype, f)
        B.check(B.nfft_grad(self.handle, _ptr(f), _ptr(cot), _ptr(out)), "nfft_grad")
        return out

    def sync(self):
        B.check(B.nfft_plan_sync(self.handle), "nfft_plan_sync")

    def info(self):
        s, nt, tile, n_items = B.nfft_plan_info(self.handle)
        B.check(s, "nfft_plan_info")
        return {"Ntilde": nt[:self.D], "tile": tile[:self.D], "n_items": n_items}

    def set_tile(self, tile):
        B.check(B.nfft_plan_set_tile(self.handle, tile), "nfft_plan_set_tile")
        self._nodes_key = None

    def autotune(self, k):
        """Choose the tile shape by timing candidates on these nodes (leaves them set)."""
        self._check_tensor(k, (self.M, self.D), k.dtype, "k")
        s, tile = B.nfft_plan_autotune(self.handle, _ptr(k), k.dtype == torch.float64)
        B.check(s, "nfft_plan_autotune")
        self._nodes_key = (k.data_ptr(), k._version, k.device)
        return tile[:self.D]

    @property
    def Ntilde(self):
        return self.info()["Ntilde"]

    def grid_tensor(self):
        """The plan's oversampled grid as a tensor view (no copy)."""
        nt = self.Ntilde
        ptr = B.nfft_plan_grid(self.handle)
        return _view_device_memory(ptr, nt, self.dtype, self.device)

    # individual steps (device tensors)
    def step_deconv_pad(self, f):
        self._check_tensor(f, self.N, self.dtype, "f")
        B.check(B.nfft_step_deconv_pad(self.handle, _ptr(f)), "nfft_step_deconv_pad")

    def step_fft(self, sign):
        B.check(B.nfft_step_fft(self.handle, sign), "nfft_step_fft")

    def step_gather(self, out):
        self._check_tensor(out, (self.M,), self.dtype, "out")
        B.check(B.nfft_step_gather(self.handle, _ptr(out)), "nfft_step_gather")
        return out

    def step_scatter(self, fhat):
        self._check_tensor(fhat, (self.M,), self.dtype, "fhat")
        B.check(B.nfft_step_scatter(self.handle, _ptr(fhat)), "nfft_step_scatter")

    def step_crop_deconv(self, out):
        self._check_tensor(out, self.N, self.dtype, "out")
        B.check(B.nfft_step_crop_deconv(self.handle, _ptr(out)), "nfft_step_crop_deconv")
        return out

    def step_pad_fft(self, f):
        """Algorithm 1's correction, zero-pad and FFT steps (the pruned FFT or
        the direct sums where the plan qualifies)."""
        self._check_tensor(f, self.N, self.dtype, "f")
        B.check(B.nfft_step_pad_fft(self.handle, _ptr(f)), "nfft_step_pad_fft")

    def step_fft_crop(self, out):
        """Algorithm 2's inverse FFT, crop and correction steps (the pruned FFT
        or the direct sums where the plan qualifies)."""
        self._check_tensor(out, self.N, self.dtype, "out")
        B.check(B.nfft_step_fft_crop(self.handle, _ptr(out)), "nfft_step_fft_crop")
        return out

    def set_graph(self, enable=True):
        """Replay nfft_forward / nfft_adjoint from captured CUDA graphs (device buffers)."""
        B.check(B.nfft_plan_set_graph(self.handle, enable), "nfft_plan_set_graph")

    def set_async(self, enable=True):
        """Host-buffer nfft_forward / nfft_adjoint return once enqueued, with
        their copies overlapping the previous call's kernels; results are
        ready after sync()."""
        B.check(B.nfft_plan_set_async(self.handle, enable), "nfft_plan_set_async")

    def paths(self):
        """{'fast_gather', 'fast_scatter', 'pruned_fft', 'fft_form'}: which
        specialised kernels this plan's transforms run (fft_form: 'library',
        'pruned' or 'direct')."""
        s, fg, fs, form = B.nfft_plan_paths(self.handle)
        B.check(s, "nfft_plan_paths")
        return {"fast_gather": fg, "fast_scatter": fs, "pruned_fft": form == 1,
                "fft_form": ("library", "pruned", "direct")[form]}

    def step_grad_gather(self, cot, out):
        self._check_tensor(cot, (self.M,), self.dtype, "cot")
        self._check_tensor(out, (self.M, self.D), self.real_dtype, "out")
        B.check(B.nfft_step_grad_gather(self.handle, _ptr(cot), _ptr(out)), "nfft_step_grad_gather")
        return out


class Batch:
    """Many NFFTs in one launch per step (nfft_batch_*): problems with their own
    sizes N[p] on node sets set_of[p] with M_set[s] nodes."""

    def __init__(self, Ns, set_of, M_set, sigma=2.0, m=4, dtype=torch.complex64, flags=0, stream=None):
        if dtype not in _DTYPES:
            raise TypeError("dtype must be torch.complex64 or torch.complex128")
        self.Ns = [tuple(int(v) for v in n) for n in Ns]
        self.D = len(self.Ns[0])
        self.set_of = [int(v) for v in set_of]
        self.M_set = [int(v) for v in M_set]
        self.dtype = dtype
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        flat = [v for n in self.Ns for v in n]
        s, h = B.nfft_batch_create(self.D, flat, self.set_of, self.M_set, sigma, m, _DTYPES[dtype], flags,
                                   self.stream.cuda_stream)
        B.check(s, "nfft_batch_create")
        self._h = h
        self.in_sizes = [int(torch.tensor(n).prod()) for n in self.Ns]
        self.out_sizes = [self.M_set[p] for p in self.set_of]

    def close(self):
        if getattr(self, "_h", None):
            B.nfft_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_nodes(self, k_all):
        """k_all: the node sets concatenated, (sum M_set, D) float64 on the device."""
        B.check(B.nfft_batch_set_nodes(self._h, _ptr(k_all), k_all.dtype == torch.float64), "nfft_batch_set_nodes")

    def forward(self, f_all, out=None):
        """f_all: concatenated flattened coefficient arrays; returns concatenated fhat."""
        if out is None:
            out = torch.empty(sum(self.out_sizes), dtype=self.dtype, device=self.device)
        B.check(B.nfft_batch_forward(self._h, _ptr(f_all), _ptr(out)), "nfft_batch_forward")
        return out

    def adjoint(self, fhat_all, out=None):
        if out is None:
            out = torch.empty(sum(self.in_sizes), dtype=self.dtype, device=self.device)
        B.check(B.nfft_batch_adjoint(self._h, _ptr(fhat_all), _ptr(out)), "nfft_batch_adjoint")
        return out

    def set_graph(self, enable=True):
        B.check(B.nfft_batch_set_graph(self._h, enable), "nfft_batch_set_graph")

    def set_tile(self, tile):
        B.check(B.nfft_batch_set_tile(self._h, tile), "nfft_batch_set_tile")

    def autotune(self, k_all):
        s, tile = B.nfft_batch_autotune(self._h, _ptr(k_all), k_all.dtype == torch.float64)
        B.check(s, "nfft_batch_autotune")
        return tile[:self.D]

    def info(self):
        s, tile, n_items, n_cls = B.nfft_batch_info(self._h)
        B.check(s, "nfft_batch_info")
        return {"tile": tile[:self.D], "n_items": n_items, "fft_classes": n_cls}


def _view_device_memory(ptr, shape, dtype, device):
    """Wrap plan-owned device memory as a tensor without copying."""
    nbytes = 1
    for s in shape:
        nbytes *= int(s)
    nbytes *= torch.empty((), dtype=dtype).element_size()

    class _Holder:
        pass

    holder = _Holder()
    holder.__cuda_array_interface__ = {
        "shape": tuple(int(s) for s in shape),
        "typestr": "<c8" if dtype == torch.complex64 else "<c16",
        "data": (int(ptr), False),
        "version": 3,
        "strides": None,
    }
    with torch.cuda.device(device):
        return torch.as_tensor(holder, device=device)


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
def _ensure_nodes(plan, k):
    if not plan.nodes_match(k):
        plan.set_nodes(k.detach().contiguous())


class _NFFTFunction(torch.autograd.Function):
    """fhat = A(k) f; grads: f -> A^H G, k -> Re(conj(G) dA f/dk)."""

    @staticmethod
    def forward(ctx, f, k, plan):
        _ensure_nodes(plan, k)
        fhat = plan.forward(f.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(f, k)
        return fhat

    @staticmethod
    def backward(ctx, G):
        plan = ctx.plan
        f, k = ctx.saved_tensors
        _ensure_nodes(plan, k)
        G = G.contiguous()
        gf = plan.adjoint(G) if ctx.needs_input_grad[0] else None
        gk = plan.grad(f.contiguous(), G).to(k.dtype) if ctx.needs_input_grad[1] else None
        return gf, gk, None


class _NFFTAdjointFunction(torch.autograd.Function):
    """y = A(k)^H w; grads: w -> A Y, k -> Re(conj(w) dA Y/dk)."""

    @staticmethod
    def forward(ctx, w, k, plan):
        _ensure_nodes(plan, k)
        y = plan.adjoint(w.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(w, k)
        return y

    @staticmethod
    def backward(ctx, Y):
        plan = ctx.plan
        w, k = ctx.saved_tensors
        _ensure_nodes(plan, k)
        Y = Y.contiguous()
        gw = plan.forward(Y) if ctx.needs_input_grad[0] else None
        gk = plan.grad(Y, w.contiguous()).to(k.dtype) if ctx.needs_input_grad[1] else None
        return gw, gk, None


def nfft(f, k, plan):
    """Differentiable direct NFFT: fhat = A(k) f."""
    return _NFFTFunction.apply(f, k, plan)


def nfft_adjoint(w, k, plan):
    """Differentiable adjoint NFFT: y = A(k)^H w."""
    return _NFFTAdjointFunction.apply(w, k, plan)
