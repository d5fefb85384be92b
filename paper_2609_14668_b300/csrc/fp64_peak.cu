// B300 microbenchmarks behind the FP64 roofline and the launch-schedule design:
// FP64 DFMA throughput and dependent latency, FP64 DMMA (mma.sync m8n8k4)
// throughput, FP32 FFMA throughput, grid-barrier latency of a cooperative
// launch (bounded spin), back-to-back launch cost.  Standalone binary:
//   python -m paper_2609_14668_b300.build --peak && paper_2609_14668_b300/fp64_peak
#include <cstdio>
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA err %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

__global__ void k_dfma(double* out, int iters, double a, double b){
  double x0=threadIdx.x*1e-3, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int i=0;i<iters;i++){
    x0=fma(x0,a,b); x1=fma(x1,a,b); x2=fma(x2,a,b); x3=fma(x3,a,b);
    x4=fma(x4,a,b); x5=fma(x5,a,b); x6=fma(x6,a,b); x7=fma(x7,a,b);
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void k_ffma(float* out, int iters, float a, float b){
  float x[16];
  for(int j=0;j<16;j++) x[j]=threadIdx.x*1e-3f+j;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int j=0;j<16;j++) x[j]=fmaf(x[j],a,b);
  }
  float s=0; for(int j=0;j<16;j++) s+=x[j];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void k_dmma(double* out, int iters){
  double a=1.0+threadIdx.x*1e-6, b=0.999;
  double c0[2]={0,0}, c1[2]={0,0}, c2[2]={0,0}, c3[2]={0,0};
  for(int i=0;i<iters;i++){
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c0[0]),"+d"(c0[1]) : "d"(a),"d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c1[0]),"+d"(c1[1]) : "d"(a),"d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c2[0]),"+d"(c2[1]) : "d"(a),"d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c3[0]),"+d"(c3[1]) : "d"(a),"d"(b));
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=c0[0]+c0[1]+c1[0]+c1[1]+c2[0]+c2[1]+c3[0]+c3[1];
}
// single-thread dependent DFMA latency chain
__global__ void k_dlat(double* out, int iters, double a, double b){
  double x=threadIdx.x;
  for(int i=0;i<iters;i++) x=fma(x,a,b);
  out[threadIdx.x]=x;
}
// grid barrier: sense via generation counter, bounded spin
__device__ unsigned int g_count=0, g_gen=0;
__global__ void k_gridbar(int nbar, int* err){
    for(int it=0; it<nbar; it++){
    __syncthreads();
    if(threadIdx.x==0){
      unsigned int my = *(volatile unsigned int*)&g_gen;
      __threadfence();
      unsigned int arrived = atomicAdd(&g_count,1);
      if(arrived==gridDim.x-1){ g_count=0; __threadfence(); atomicAdd(&g_gen,1);} 
      else { long long spin=0; while(*(volatile unsigned int*)&g_gen==my){ if(++spin>(1ll<<26)){ atomicExch(err,1); break;} } }
      __threadfence();
    }
    __syncthreads();
  }
}
int main(){
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev)); int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("GPU %s SMs %d cc %d.%d clock %d kHz smemPerBlockOptin %zu L2 %d\n", p.name, p.multiProcessorCount, p.major, p.minor, clk, p.sharedMemPerBlockOptin, p.l2CacheSize);
  int sms=p.multiProcessorCount;
  double* dout; float* fout; int* derr; CK(cudaMalloc(&dout, 1<<24)); CK(cudaMalloc(&fout,1<<24)); CK(cudaMalloc(&derr,4)); CK(cudaMemset(derr,0,4));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for(int blocksPerSM: {4,8}){
    int iters=20000, thr=256, grid=sms*blocksPerSM;
    k_dfma<<<grid,thr>>>(dout,100,1.0000001,1e-9); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dfma<<<grid,thr>>>(dout,iters,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*8*iters*(double)grid*thr; printf("DFMA grid %d: %.3f ms  %.3f TFLOP/s\n", grid, ms, fl/ms/1e9);
  }
  { int iters=20000, thr=256, grid=sms*8;
    k_ffma<<<grid,thr>>>(fout,100,1.0000001f,1e-9f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_ffma<<<grid,thr>>>(fout,iters,1.0000001f,1e-9f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double fl=2.0*16*iters*(double)grid*thr; printf("FFMA: %.3f ms %.2f TFLOP/s\n", ms, fl/ms/1e9); }
  for(int blocksPerSM: {4,8}){ int iters=5000, thr=256, grid=sms*blocksPerSM;
    k_dmma<<<grid,thr>>>(dout,10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dmma<<<grid,thr>>>(dout,iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double fl=2.0*8*8*4*4*(double)iters*grid*(thr/32); printf("DMMA grid %d: %.3f ms %.3f TFLOP/s\n", grid, ms, fl/ms/1e9); }
  { int iters=100000; k_dlat<<<1,1>>>(dout,10,1.0,1e-9); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dlat<<<1,1>>>(dout,iters,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("DFMA dependent latency: %.2f ns/op (%.1f clk at %d MHz)\n", ms*1e6/iters, ms*1e6/iters*clk/1e6, clk/1000);
    for(int w: {1,32}){ cudaEventRecord(e0); k_dlat<<<1,w>>>(dout,iters,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1); printf("  %d threads: %.2f ns/op\n", w, ms*1e6/iters);} }
  for(int grid: {16, 74, 148}){
    int nbar=20000; void* args[]={&nbar,&derr};
    CK(cudaLaunchCooperativeKernel((void*)k_gridbar, grid, 128, args, 0, 0)); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); CK(cudaLaunchCooperativeKernel((void*)k_gridbar, grid, 128, args, 0, 0)); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); int herr; cudaMemcpy(&herr,derr,4,cudaMemcpyDeviceToHost);
    printf("grid barrier (%d CTAs): %.3f us/barrier err=%d\n", grid, ms*1e3/nbar, herr);
  }
  // empty-kernel launch overhead
  { cudaEventRecord(e0); for(int i=0;i<2000;i++) k_dlat<<<1,1>>>(dout,1,1.0,0.0); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1); printf("back-to-back tiny launches: %.2f us each\n", ms*1e3/2000);}  
  return 0;
}
