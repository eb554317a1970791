// Unit-rate and accuracy probe for the roofline of the far kernel: MUFU (rsqrt, sin, cos, ex2)
// and FFMA/FFMA2 lane-ops per clock per SM via clock64(), and the absolute error of
// sin.approx/cos.approx against FP64 over argument ranges.  In-bounds, no waits.
#include <cstdio>
#include <cmath>
#include <cuda_runtime.h>
__device__ __forceinline__ float rsq(float x){float y;asm volatile("rsqrt.approx.ftz.f32 %0,%1;":"=f"(y):"f"(x));return y;}
__device__ __forceinline__ float sn(float x){float y;asm volatile("sin.approx.ftz.f32 %0,%1;":"=f"(y):"f"(x));return y;}
__device__ __forceinline__ float cs(float x){float y;asm volatile("cos.approx.ftz.f32 %0,%1;":"=f"(y):"f"(x));return y;}
__device__ __forceinline__ float ex2(float x){float y;asm volatile("ex2.approx.ftz.f32 %0,%1;":"=f"(y):"f"(x));return y;}
__device__ __forceinline__ float rcp(float x){float y;asm volatile("rcp.approx.ftz.f32 %0,%1;":"=f"(y):"f"(x));return y;}
constexpr int IT = 2048, CH = 8;
template<int OP> __global__ void tput(float* out, long long* cyc){
  float x[CH];
  for(int i=0;i<CH;++i) x[i]=1.0f+0.001f*(threadIdx.x+i);
  float2 p[CH]; for(int i=0;i<CH;++i) p[i]=make_float2(x[i],x[i]+1.f);
  const float2 a2=make_float2(0.999f,0.999f), b2=make_float2(0.001f,0.001f);
  __syncthreads();
  long long t0=clock64();
  for(int it=0;it<IT;++it){
    #pragma unroll
    for(int i=0;i<CH;++i){
      if(OP==0) x[i]=rsq(x[i]);
      else if(OP==1) x[i]=sn(x[i]);
      else if(OP==2) x[i]=cs(x[i]);
      else if(OP==3) x[i]=ex2(x[i]);
      else if(OP==4) x[i]=fmaf(x[i],0.999f,0.001f);
      else if(OP==5) p[i]=__ffma2_rn(p[i],a2,b2);
      else if(OP==6) x[i]=rcp(x[i]);
    }
  }
  long long t1=clock64();
  __syncthreads();
  float s=0; for(int i=0;i<CH;++i) s+=x[i]+p[i].x+p[i].y;
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
  if(threadIdx.x==0) cyc[blockIdx.x]=t1-t0;
}
__global__ void acc(const float* xs, int n, float* es, float* ec){
  int i=blockIdx.x*blockDim.x+threadIdx.x; if(i>=n) return;
  float x=xs[i]; es[i]=fabsf(sn(x)-(float)sin((double)x)); ec[i]=fabsf(cs(x)-(float)cos((double)x));
}
int main(){
  int dev=0; cudaDeviceProp pr; cudaGetDeviceProperties(&pr,dev);
  int sms=pr.multiProcessorCount; printf("SMs %d\n",sms);
  const char* names[]={"rsqrt","sin","cos","ex2","ffma","ffma2","rcp"};
  for(int bs: {256,512}){
   int blocks=sms*(2048/bs);
   float* out; long long* cyc; cudaMalloc(&out,sizeof(float)*blocks*bs); cudaMalloc(&cyc,sizeof(long long)*blocks);
   long long* h=new long long[blocks];
   for(int op=0;op<7;++op){
    for(int rep=0;rep<2;++rep){
    switch(op){case 0:tput<0><<<blocks,bs>>>(out,cyc);break;case 1:tput<1><<<blocks,bs>>>(out,cyc);break;case 2:tput<2><<<blocks,bs>>>(out,cyc);break;
      case 3:tput<3><<<blocks,bs>>>(out,cyc);break;case 4:tput<4><<<blocks,bs>>>(out,cyc);break;case 5:tput<5><<<blocks,bs>>>(out,cyc);break;case 6:tput<6><<<blocks,bs>>>(out,cyc);break;}
    cudaError_t e=cudaDeviceSynchronize(); if(e){printf("err %s\n",cudaGetErrorString(e));return 1;}
    }
    cudaMemcpy(h,cyc,sizeof(long long)*blocks,cudaMemcpyDeviceToHost);
    double mx=0; for(int b=0;b<blocks;++b) mx=h[b]>mx?h[b]:mx;
    double ops_per_sm=(double)(2048/bs)*bs*IT*CH*(op==5?2:1);
    printf("bs=%d %-6s lane-ops/clk/SM %.1f (max cycles %.0f)\n",bs,names[op],ops_per_sm/mx,mx);
   }
   cudaFree(out);cudaFree(cyc);delete[] h;
  }
  const int n=1<<22; float* xs; float *es,*ec; cudaMallocManaged(&xs,n*4); cudaMallocManaged(&es,n*4); cudaMallocManaged(&ec,n*4);
  for(int i=0;i<n;++i) xs[i]=(float)(i*(400.0/n));
  acc<<<(n+255)/256,256>>>(xs,n,es,ec); cudaDeviceSynchronize();
  double edges[]={0,3.1416,31.416,100,157.08,200,314.16,400.01};
  for(int b=0;b<7;++b){double ms=0,mc=0; for(int i=0;i<n;++i) if(xs[i]>=edges[b]&&xs[i]<edges[b+1]){ms=es[i]>ms?es[i]:ms;mc=ec[i]>mc?ec[i]:mc;}
    printf("x in [%.1f,%.1f): max|sin err| %.3e  max|cos err| %.3e\n",edges[b],edges[b+1],ms,mc);}
  return 0;
}
