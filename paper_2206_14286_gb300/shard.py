"""N-sharded search: a database split by rows over several GPUs, one process
per GPU (Sec. 7; App. A.1's reduction_input_size_override). Argument
marshalling and the two exchanges only: PartialReduce, ExactRescoring, the
FP32 scoring and the final top-K run in libtpuknn.so (knn_shard_*).

Every shard holds global rows [row0, row0 + n); bins are j mod L of the
global row index with L planned for the whole database, and every row0 is a
multiple of L (shard_bounds), so a shard's rows keep their global bins. The
search of one query batch:
  1. each shard: PartialReduce of its rows -> M x L signed-order keys;
  2. exchange 1: element-wise MAX over the shards (all-reduce) -> the bin
     winners of the whole database, the same on every shard;
  3. each shard: ExactRescoring's top Kp of them, and the FP32 scores of the
     candidates whose rows it holds -> M x Kp keys (empty for the others);
  4. exchange 2: element-wise MAX -> every candidate's FP32 score;
  5. the best K per query (any shard; all get the same answer).
"""
import torch

from . import _lib
from ._lib import METRIC, check
from .search import Database, _stream, _workspace


def shard_bounds(N, shards, L):
    """[(row0, n)] for `shards` shards of an N-row database: starts at
    multiples of L, sizes as even as that allows, every shard at least L rows
    (ValueError otherwise)."""
    if shards < 1 or L < 1 or N < 1:
        raise ValueError("need N, shards, L >= 1")
    per = -(-N // shards)
    per = -(-per // L) * L
    out = []
    for r in range(shards):
        row0 = r * per
        n = min(per, N - row0)
        if n < L:
            raise ValueError("shard %d would hold %d rows, fewer than L = %d" % (r, max(n, 0), L))
        out.append((row0, n))
    return out


def sharded_search(shard, q, K, L, rerank, allreduce_max):
    """The search of one shard: shard.partial / rescore / finish with the two
    exchanges in between; allreduce_max(t) merges the int64 tensor t in place
    by an element-wise maximum over all shards (identity for one shard)."""
    keys = shard.partial(q, L)
    allreduce_max(keys)
    cand = shard.rescore(keys, q, K, rerank, L)
    allreduce_max(cand)
    return shard.finish(cand, K)


def dist_allreduce_max(group=None):
    """allreduce_max over a torch.distributed process group (NCCL for CUDA
    tensors, gloo for CPU tensors); the identity when the group has one rank."""
    import torch.distributed as dist

    def ar(t):
        if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return ar


class DatabaseShard:
    """Global rows [row0, row0 + n) of an N_global-row database, prepared on
    this GPU. x_local: n x D float32 CUDA rows."""

    def __init__(self, x_local, row0, N_global, metric="l2", dtype="bf16"):
        self.db = Database(x_local, metric=metric, dtype=dtype, keep_f32=True)
        self.row0, self.N_global = int(row0), int(N_global)
        self.n, self.D = self.db.N, self.db.D
        self.metric, self.dtype, self.device = metric, dtype, self.db.device
        self._ws = {}

    def _buf(self, key, nbytes):
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = _workspace(nbytes, self.device)
            self._ws[key] = ws
        return ws

    def partial(self, q, L, stream=None):
        q = q.contiguous()
        M = q.shape[0]
        lib = _lib.get()
        d = self.db
        nb = lib.knn_shard_partial_reduce_workspace(self.n, self.row0, self.N_global, self.D,
                                                    _lib.DTYPE[self.dtype], METRIC[self.metric],
                                                    M, L)
        if nb == 0:
            raise ValueError("invalid shard (row0=%d n=%d N=%d L=%d)"
                             % (self.row0, self.n, self.N_global, L))
        ws = self._buf("partial", nb)
        keys = torch.empty((M, L), dtype=torch.int64, device=self.device)
        a = d._args()
        with torch.cuda.device(self.device):
            check(lib.knn_shard_partial_reduce(a[0], a[1], a[2], self.n, self.row0, self.N_global,
                                               self.D, a[6], a[7], q.data_ptr(), M, L,
                                               keys.data_ptr(), ws.data_ptr(), ws.numel(),
                                               _stream(stream)), "knn_shard_partial_reduce")
        return keys

    def rescore(self, keys, q, K, rerank, L, stream=None):
        q = q.contiguous()
        M = q.shape[0]
        lib = _lib.get()
        Kp = lib.knn_rescore_count(K, rerank, L)
        nb = lib.knn_shard_rescore_workspace(M, L, self.D, METRIC[self.metric], K, rerank)
        if Kp < 1 or nb == 0:
            raise ValueError("invalid rescoring arguments (K=%d L=%d)" % (K, L))
        ws = self._buf("rescore", nb)
        cand = torch.empty((M, Kp), dtype=torch.int64, device=self.device)
        with torch.cuda.device(self.device):
            check(lib.knn_shard_rescore(keys.data_ptr(), M, L, K, rerank, q.data_ptr(), self.D,
                                        METRIC[self.metric], self.db.f32.data_ptr(), self.n,
                                        self.row0, cand.data_ptr(), ws.data_ptr(), ws.numel(),
                                        _stream(stream)), "knn_shard_rescore")
        return cand

    def finish(self, cand, K, stream=None):
        M, Kp = cand.shape
        lib = _lib.get()
        nb = lib.knn_shard_finish_workspace(M, Kp, K)
        if nb == 0:
            raise ValueError("invalid finish arguments (Kp=%d K=%d)" % (Kp, K))
        ws = self._buf("finish", nb)
        val = torch.empty((M, K), dtype=torch.float32, device=self.device)
        idx = torch.empty((M, K), dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            check(lib.knn_shard_finish(cand.data_ptr(), M, Kp, K, METRIC[self.metric],
                                       val.data_ptr(), idx.data_ptr(), ws.data_ptr(), ws.numel(),
                                       _stream(stream)), "knn_shard_finish")
        return val, idx

    def search(self, q, K, L, rerank=2, group=None):
        """The sharded search over a process group (every rank calls it with
        the same queries); returns (values, indices) M x K on every rank."""
        return sharded_search(self, q, K, L, rerank, dist_allreduce_max(group))
