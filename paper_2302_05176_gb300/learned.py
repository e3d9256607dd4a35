"""The learned first-pass bound: training set, training loop and the model object.

Every step runs in libgm's kernels (gm_features, gm_row_ln_ystar,
gm_model_grad, gm_model_adam, gm_sketch_learned); this module only sequences the
calls.  The target of each row is ln y*, the log of its largest register, taken
from exact sketches of synthetic rows; the network is fitted to the tau-quantile
of ln y* given the row features (pinball loss), so its bound exp(prediction)
covers y* in a fraction tau of rows and the rest fall back to the closed-form
bound of the second pass.

Because y* Sum(v) follows the law of the largest of k independent Exp(1)
variables for every weight vector, the features beyond (ln Sum v, ln k) carry no
information about y*: the best the network can do is the closed-form quantile
-ln(1 - tau^(1/k)) / Sum(v).  The fallback rate of the trained model is
therefore expected to be close to 1 - tau, and its work close to the closed-form
bound's; what it gains over FastGM without an initial bound is measured.
"""
import math
from dataclasses import dataclass, field

import torch

from . import gm
from .workloads import lognormal_batch_device, single_vector_batch_device


@dataclass
class TrainingSet:
    feats: torch.Tensor   # [N, 8] float32, device
    target: torch.Tensor  # [N] float32, ln y*
    ks: list = field(default_factory=list)


LAWS = {"lognormal": lognormal_batch_device, "single_vector": single_vector_batch_device}


def make_training_set(n_sketches=200_000, ks=(256, 1024, 4096), seed=1000, rows_per_batch=4096, device="cuda",
                      law="lognormal"):
    """Sketch n_sketches synthetic rows (law "lognormal": the lognormal_batch
    distribution; "single_vector": rows of n+ = 1,000 of 10,000 dimensions with
    Uniform(0,1] weights; the k values taken in turn per batch) with gm_sketch and
    keep (features, ln y*)."""
    draw = LAWS[law]
    feats, target, klist = [], [], []
    done, b = 0, 0
    while done < n_sketches:
        n = min(rows_per_batch, n_sketches - done)
        k = int(ks[b % len(ks)])
        row_ptr, ids, w = draw(seed + b, n_rows=n, device=device)
        _, y, ws = gm.gm_sketch(row_ptr, ids, w, k, seed + 7919 * b)
        t = gm.gm_row_ln_ystar(y)
        f = gm.gm_features(row_ptr, ids, w, k)
        ok = torch.isfinite(t)
        feats.append(f[ok])
        target.append(t[ok])
        klist.append(k)
        del ws, y
        done += n
        b += 1
    return TrainingSet(torch.cat(feats), torch.cat(target), klist)


def train(ts, tau=0.95, steps=400, lr=3e-3, lr_final=1e-4, seed=7, device="cuda", log_every=0):
    """Full-batch Adam on the mean pinball loss; cosine decay lr -> lr_final.
    Returns (params, [loss at each logged step])."""
    params = gm.gm_model_init(seed, device=device)
    adam = torch.zeros(2 * gm.GM_MODEL_PARAMS, dtype=torch.float32, device=params.device)
    grad = torch.empty(gm.GM_MODEL_PARAMS, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    ws = torch.empty(gm.gm_model_grad_workspace_bytes(), dtype=torch.uint8, device=params.device)
    history = []
    for step in range(1, steps + 1):
        gm.gm_model_grad(params, ts.feats, ts.target, tau, grad=grad, loss=loss, ws=ws)
        c = 0.5 * (1.0 + math.cos(math.pi * (step - 1) / max(1, steps - 1)))
        gm.gm_model_adam(params, adam, grad, lr_final + (lr - lr_final) * c, step)
        if log_every and (step % log_every == 0 or step == steps):
            history.append((step, float(loss.item())))
    gm.gm_model_grad(params, ts.feats, ts.target, tau, grad=grad, loss=loss, ws=ws)
    history.append((steps + 1, float(loss.item())))
    return params, history


class BoundModel:
    """A trained network plus the margin added to its ln y* prediction."""

    def __init__(self, params, margin=0.0, tau=None):
        self.params = params
        self.margin = float(margin)
        self.tau = tau

    @classmethod
    def load(cls, path, margin=0.0, device="cuda"):
        return cls(gm.gm_model_load(path, device=device), margin)

    def save(self, path):
        gm.gm_model_save(self.params, path)

    def predict(self, feats):
        return gm.gm_model_forward(self.params, feats)

    def sketch(self, row_ptr, ids, w, k, seed, flags=0, s_out=None, y_out=None, ws=None, stream=None):
        return gm.gm_sketch_learned(row_ptr, ids, w, k, seed, self.params, self.margin, flags, s_out, y_out, ws,
                                    stream)
