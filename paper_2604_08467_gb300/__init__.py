"""GB300-native tensor-network PTSBE hot path (arxiv 2604.08467).

The compute path lives in ``libptn.so`` (CUDA for sm_103a, C ABI in
``include/ptn.h``); ``ptn`` is its thin ctypes binding and ``autograd`` wraps
``ptn_expval_grad`` as a torch.autograd.Function.
"""
from .ptn import (PtnError, Plan, Shots, Traj, ptn_allocate_shots, ptn_contract_batch,  # noqa: F401
                  ptn_expval_grad, ptn_plan_path, ptn_presample_trajectories, ptn_sample_block,
                  ptn_sample_shots)
