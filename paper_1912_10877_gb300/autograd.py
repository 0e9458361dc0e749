"""torch.autograd.Function around expect'(O, zero_state => circuit) (Sec. "Reverse Mode").

Forward: |0...0> (or a basis state) -> circuit -> <O>, optionally saving
checkpoints every ``ckpt_every`` gates.  Backward: the library's reversible
adjoint kernel uncomputes the saved output state and returns dL/dparams.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qsim


class CircuitExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, circuit, observable, dtype=torch.complex64, ckpt_every=0, basis=0):
        p = params.detach().to("cpu", torch.float64).numpy()
        st = qsim.State(circuit.nqubits, dtype=dtype)
        st.reset([basis])
        ckpts = qsim.checkpoint_buffer(st, circuit, ckpt_every) if ckpt_every else None
        if ckpt_every:
            qsim.apply_circuit_ckpt(st, circuit, p, ckpt_every, ckpts)
        else:
            st.apply_circuit(circuit, p)
        loss = float(st.expect(observable)[0])
        ctx.state, ctx.circuit, ctx.observable = st, circuit, observable
        ctx.p, ctx.ckpt_every, ctx.ckpts = p, ckpt_every, ckpts
        return params.new_tensor(loss)

    @staticmethod
    def backward(ctx, grad_out):
        _, g = qsim.backward(ctx.state, ctx.circuit, ctx.p, ctx.observable, ctx.ckpt_every, ctx.ckpts)
        g = torch.as_tensor(np.asarray(g), dtype=grad_out.dtype, device=grad_out.device) * grad_out
        ctx.state = ctx.ckpts = None
        return g, None, None, None, None, None


def expectation(params: torch.Tensor, circuit, observable, dtype=torch.complex64, ckpt_every=0, basis=0):
    return CircuitExpectation.apply(params, circuit, observable, dtype, ckpt_every, basis)
